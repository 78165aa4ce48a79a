// Gram matrix G = X^T Y of the Rayleigh-Ritz step (Step 4, eq. 3.3) on the
// 5th-generation tensor cores (tcgen05), for the mixed path with Np <= kTcMaxNp.
//
// X and Y arrive as the float32 hi parts of the float-float arrays [node][Np]
// (each the float64 value rounded to the nearest float, an unbiased rounding).
// The products are made exact so that the FP32 accumulator of the tensor cores
// never rounds:
//   * per CTA, chunk of kTcSuper = 128 nodes and column c, E_c is the power of
//     two above max |x_c| over the chunk (a scale that follows the local size);
//   * every value becomes three signed integer digits, x = 2^E_c (s0 2^-8 +
//     s1 2^-16 + s2 2^-24) + r, each digit the nearest integer to the scaled
//     remainder (|s0| <= 256, |s1|, |s2| <= 128, |r| <= 2^(E_c - 25)); integers
//     of this size are exact in BF16;
//   * the digit products of one level l = i + j (i, j digit indices, l <= 2)
//     go to their own FP32 accumulator in tensor memory: a product is an integer
//     below 2^16 and a level's sum over kTcSuper = 128 nodes stays below 2^24, so
//     every partial sum is an exact integer in FP32 whatever the order of
//     accumulation;
//   * per chunk the three levels are combined into a float-float value, scaled
//     by 2^(E_a + E_b) and added to float-float accumulators.
// The error is the rounding of the inputs to 24 bits below the chunk's column
// maximum (the digit rounding and the dropped lo part, together <= 2^(E_c - 24)
// per value, both to nearest and so unbiased), so it averages out over the
// nodes: about
// 2^-24 / sqrt(nodes) of |x| |y| for a Gram entry, instead of the
// 2^-24-per-addition growth of a plain FP32 sum.  Levels l >= 3 (products below
// 2^-48 of the scale) are dropped.
//
// A launch computes one block of G (128 rows x 64 columns, or 32 x 32 for
// Np <= 32); larger Np are tiled over several launches.
// Per CTA: a chunk's two halves of 64 nodes are loaded into registers, their
// column maxima reduced in shared memory, and then converted into two
// shared-memory operand buffers, so the MMAs of the first half run while the
// second is converted; the next chunk's loads are in flight during the MMAs and
// the read-out.
// A thread converts 8 nodes of one orbital of X or Y into 16-byte rows (one per
// digit plane) of the canonical K-major layout without swizzle: core matrices of
// 8 rows x 16 bytes, kTcLBO = 128 bytes between core matrices along K and
// kTcSBO = 1040 bytes between 8-row groups (16 bytes of padding that spread the
// rows of one warp's stores over all banks).  One thread issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128 rows = orbital a, zero-padded;
// N = NCOL; K = 16; BF16 in, FP32 out) and commits to an mbarrier.  The
// float-float accumulators live in shared memory, [column][row] (conflict-free).  Every wait
// is bounded; on a timeout the CTA records kStatTimeout, waits once more
// (bounded) for its MMAs, frees its tensor memory and returns.  Each CTA writes
// its partial G in float64 for the fixed-order reduction of rr.cu.
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "ff.cuh"
#include "tma.cuh"

namespace paro {

namespace {

constexpr int kTcHalf = 64;    // nodes per operand buffer (4 K-steps of 16)
constexpr int kTcSuper = 128;  // nodes per exact accumulation (two buffers)
constexpr int kTcM = 128;      // MMA rows (orbital a, zero-padded)
constexpr int kTcDigits = 3;   // digits per value = accumulation levels
constexpr int kTcLBO = 128;    // bytes between core matrices along K
constexpr int kTcSBO = 1040;   // bytes between 8-row groups (8 core matrices + 16 bytes of padding)
constexpr int kTcEmin = -100, kTcEmax = 100;  // range of the column exponents

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start address, leading / stride byte offsets (>> 4), version 1 (bits 46-47),
  // base offset 0, no swizzle
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of the 16-byte row segment (row, nodes 8 k8 .. 8 k8 + 7) of an operand plane.
__device__ __forceinline__ uint32_t op_off(int row, int k8) {
  return (uint32_t)((row >> 3) * kTcSBO + k8 * kTcLBO + (row & 7) * 16);
}

// 2^e as a float, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Signed digits of x * s256 / 256 (|x * s256| < 256): d_k = the nearest integer to
// 256^k x the remainder left by the digits before it; every step is exact.
__device__ __forceinline__ void digits3(float x, float s256, float (&d)[kTcDigits]) {
  float a = __fmul_rn(x, s256);
#pragma unroll
  for (int k = 0; k < kTcDigits; ++k) {
    d[k] = rintf(a);
    a = __fmul_rn(__fsub_rn(a, d[k]), 256.0f);
  }
}

__device__ __forceinline__ int col_exponent(unsigned bits) {
  // smallest E with max |x| < 2^E (bits: the float bit pattern of max |x|)
  if (bits == 0u) return 0;
  int e = (int)(bits >> 23) - 126;
  return e < kTcEmin ? kTcEmin : (e > kTcEmax ? kTcEmax : e);
}



__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);  // exact: integers below 2^8 in magnitude (or 256)
  return *reinterpret_cast<const uint32_t*>(&p);
}

constexpr int kTcThreads = 512;

template <int NCOL>
__host__ __device__ constexpr int tc_buf_bytes() {
  return kTcDigits * ((kTcM / 8) * kTcSBO + (NCOL / 8) * kTcSBO);
}
// dynamic shared memory: two operand buffers, then the float-float accumulators [NCOL][128]
template <int NCOL>
__host__ __device__ constexpr int tc_smem_bytes() {
  return 2 * tc_buf_bytes<NCOL>() + NCOL * kTcM * (int)sizeof(FF);
}

// One block of G: rows a = xr0 .. xr0 + na - 1 (na <= 128, the MMA's M side) and
// columns b = yc0 .. yc0 + nb - 1 (nb <= NCOL = 32 or 64, the MMA's N side) of
// G = X^T Y, X and Y [node][Np].  For the read-out warp w takes TMEM lanes
// 32 (w % 4) .. and the column group w / 4 (of 4).
// Two Grams in one launch (yh2 != null): columns b < nb1 from yh (G = X^T Y into
// part), b >= nb1 from yh2 (X^T Y2 into part2): X is loaded and converted once.
template <int NCOL>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(long long G, int Np, int xr0, int na, int yc0, int nb, const float* __restrict__ xh,
              const float* __restrict__ yh, double* __restrict__ part, long long chunk, int* __restrict__ status,
              const float* __restrict__ yh2, int nb1, double* __restrict__ part2) {
  constexpr int kCols = NCOL / 4;  // columns a thread reads out
  constexpr uint32_t kTmemCols = kTcDigits * NCOL <= 128 ? 128 : 256;
  constexpr int kAPiece = (kTcM / 8) * kTcSBO;  // bytes of one A digit plane (128 rows x 64 nodes)
  constexpr int kBPiece = (NCOL / 8) * kTcSBO;  // bytes of one B digit plane
  constexpr int kBuf = tc_buf_bytes<NCOL>();
  extern __shared__ __align__(1024) unsigned char smem[];
  FF* accs = reinterpret_cast<FF*>(smem + 2 * kBuf);  // [column][row]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ float s256[kTcM + NCOL];
  __shared__ int cexp[kTcM + NCOL];       // rows a, then columns b
  __shared__ unsigned cmax[kTcM + NCOL];  // chunk maxima of |x| (float bits)
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

  // zero both operand buffers (rows beyond na / nb stay zero) and the accumulators
  for (int i = tid; i < tc_smem_bytes<NCOL>() / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < kTcM + NCOL; i += kTcThreads) {
    cexp[i] = 0;
    cmax[i] = 0u;
  }
  if (tid == 0) {
    s_fail = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  // conversion work items (array X or Y, node octet of the half, orbital), the
  // orbital fastest so that a warp's loads and 16-byte row stores are contiguous;
  // a thread takes items tid, tid + 512, ... (at most kItems)
  // (the 32-column variant serves Np <= 32 only: na, nb <= 32)
  constexpr int kItems = (8 * ((NCOL == 32 ? 32 : kTcM) + NCOL) + kTcThreads - 1) / kTcThreads;
  const int nx = 8 * na, nitems = 8 * (na + nb);
  float v[2][kItems][8];  // the chunk's two halves
  auto item = [&](int w, int& arr, int& oct, int& o) {
    arr = w >= nx;
    const int r2 = w - (arr ? nx : 0), n = arr ? nb : na;
    oct = r2 / n;
    o = r2 - oct * n;
  };
  auto load = [&](int h, long long n1, long long end) {
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const int w = tid + it * kTcThreads;
      int arr, oct, o;
      item(w, arr, oct, o);
      const float* src = !arr ? xh + xr0 + o : (o < nb1 ? yh + yc0 + o : yh2 + (o - nb1));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long node = n1 + 8 * oct + j;
        v[h][it][j] = (w < nitems && node < end) ? __ldg(src + node * Np) : 0.0f;
      }
    }
  };
  // the chunk's column maxima -> exponents and digit scales
  auto scales = [&]() {
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const int w = tid + it * kTcThreads;
      if (w < nitems) {
        int arr, oct, o;
        item(w, arr, oct, o);
        unsigned m = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j) m = max(m, __float_as_uint(v[h][it][j]) & 0x7FFFFFFFu);
        if (m != 0u) atomicMax(&cmax[arr ? kTcM + o : o], m);
      }
    }
    __syncthreads();
    for (int i = tid; i < kTcM + NCOL; i += kTcThreads) {
      const int e = col_exponent(cmax[i]);
      cexp[i] = e;
      s256[i] = pow2f(8 - e);
      cmax[i] = 0u;
    }
    __syncthreads();
  };
  auto store = [&](int h, unsigned char* buf) {
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const int w = tid + it * kTcThreads;
      if (w < nitems) {
        int arr, oct, o;
        item(w, arr, oct, o);
        const float sc = s256[arr ? kTcM + o : o];
        uint32_t q[kTcDigits][4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float d0[kTcDigits], d1[kTcDigits];
          digits3(v[h][it][j], sc, d0);
          digits3(v[h][it][j + 1], sc, d1);
#pragma unroll
          for (int p = 0; p < kTcDigits; ++p) q[p][j / 2] = pack_bf16(d0[p], d1[p]);
        }
        unsigned char* dst = buf + (arr ? kTcDigits * kAPiece : 0) + op_off(o, oct);
        const int pstep = arr ? kBPiece : kAPiece;
#pragma unroll
        for (int p = 0; p < kTcDigits; ++p)
          *reinterpret_cast<uint4*>(dst + p * pstep) = make_uint4(q[p][0], q[p][1], q[p][2], q[p][3]);
      }
    }
  };

  const int row = 32 * (warp % 4) + lane;  // orbital xr0 + row of this thread in the read-out
  const int col0 = (warp / 4) * kCols;

  const uint32_t idesc = idesc_bf16(kTcM, NCOL);
  const uint32_t sbase = smem_u32(smem);
  const long long beg = (long long)blockIdx.x * chunk;
  long long end = beg + chunk;
  if (end > G) end = G;
  uint32_t phase = 0;
  if (beg < end) {
    load(0, beg, end);
    load(1, beg + kTcHalf, end);
  }
  for (long long n0 = beg; n0 < end; n0 += kTcSuper) {
    scales();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      store(h, smem + h * kBuf);
      // the next chunk's loads are in flight during the MMAs and the read-out
      const long long nn = n0 + kTcSuper + h * kTcHalf;
      if (n0 + kTcSuper < end) load(h, nn, end);
      fence_proxy_async_smem();  // generic writes -> the MMA's async-proxy reads
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t aBase = sbase + h * kBuf, bBase = aBase + kTcDigits * kAPiece;
#pragma unroll
        for (int l = 0; l < kTcDigits; ++l) {
#pragma unroll
          for (int i = 0; i <= l; ++i) {
#pragma unroll
            for (int ks = 0; ks < kTcHalf / 16; ++ks) {
              const uint64_t ad = smem_desc(aBase + i * kAPiece + ks * 2 * kTcLBO, kTcLBO, kTcSBO);
              const uint64_t bd = smem_desc(bBase + (l - i) * kBPiece + ks * 2 * kTcLBO, kTcLBO, kTcSBO);
              mma_bf16(tmem + (uint32_t)(l * NCOL), ad, bd, idesc, (h > 0 || i > 0 || ks > 0) ? 1u : 0u);
            }
          }
        }
        if (h == 1) mma_commit(&bar);
      }
    }
    bool ok = mbar_wait(&bar, phase);
    if (!ok) {
      s_fail = 1;
      ok = mbar_wait(&bar, phase);  // let the MMAs in flight end before the memory is freed (bounded)
    }
    phase ^= 1;
    tc_fence_after();
    __syncthreads();
    if (s_fail) break;
    // combine the three exact level sums of the 128 nodes and add them to the
    // accumulators; only the warps whose TMEM lanes hold rows a < na (the rest of
    // the 128 MMA rows are zero padding: 12 of 16 warps at Np <= 32)
    const float sa = pow2f(cexp[row] - 8);
#pragma unroll
    for (int c = 0; c < kCols && 32 * (warp % 4) < na; c += 8) {
      const uint32_t ta = tmem + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(col0 + c);
      float v0[8], v1[8];
      tmem_ld8(ta, v0);
      tmem_ld8(ta + NCOL, v1);
      FF tsum[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) two_sum(v0[i], __fmul_rn(v1[i], 0x1p-8f), tsum[i].hi, tsum[i].lo);
      tmem_ld8(ta + 2 * NCOL, v0);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        ff_add(tsum[i], FF{__fmul_rn(v0[i], 0x1p-16f), 0.f});
        const int b = col0 + c + i;
        const float sc = __fmul_rn(sa, pow2f(cexp[kTcM + b] - 8));
        FF a = accs[b * kTcM + row];
        ff_add(a, FF{__fmul_rn(tsum[i].hi, sc), __fmul_rn(tsum[i].lo, sc)});
        accs[b * kTcM + row] = a;
      }
    }
    tc_fence_before();
    __syncthreads();  // every thread read the accumulators before the next chunk's MMAs
  }
  if (s_fail && tid == 0) atomicOr(status, kStatTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  // the block's partial, G[xr0 + a][yc0 + b], written row-major with coalesced columns
  const long long NN = (long long)Np * Np;
  double* dst = part + (long long)blockIdx.x * NN;
  double* dst2 = part2 ? part2 + (long long)blockIdx.x * NN : nullptr;
  for (int t = tid; t < na * nb; t += kTcThreads) {
    const int a = t / nb, b = t % nb;
    const double v = ff_to_double(ff_norm(accs[b * kTcM + a]));
    if (b < nb1) dst[(long long)(xr0 + a) * Np + yc0 + b] = v;
    else dst2[(long long)(xr0 + a) * Np + (b - nb1)] = v;
  }
}

template <int NCOL>
cudaError_t launch_tc(long long G, int Np, int xr0, int na, int yc0, int nb, const float* xh, const float* yh,
                      double* part, long long chunk, int nch, int* status, cudaStream_t st,
                      const float* yh2 = nullptr, int nb1 = 1 << 30, double* part2 = nullptr) {
  const size_t smem = (size_t)tc_smem_bytes<NCOL>();
  cudaError_t e = allow_max_dyn_smem((const void*)k_gram_tc<NCOL>);
  if (e != cudaSuccess) return e;
  k_gram_tc<NCOL><<<nch, kTcThreads, smem, st>>>(G, Np, xr0, na, yc0, nb, xh, yh, part, chunk, status, yh2, nb1,
                                                   part2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The rotation U = X C of the Rayleigh-Ritz step (Step 4) on the tensor cores,
// for Np <= kRotTcMaxNp: D[128 nodes][NB columns] = A[128 nodes][K = a] B[K = a][NB]
// with A the digits of X (the float32 hi parts, one power-of-two scale per node
// row: the row maximum over a) and B the digits of C (one scale per column b).
// Three digits each, levels l = i + j <= 2 in their own FP32 accumulators; every
// level sum over K = a <= 128 terms stays below 2^24, so it is exact.  The three
// levels are combined in float-float and scaled by 2^(E_g + F_b) in float64.
// The error is the rounding of X and C to 24 bits below their row / column
// maximum (unbiased), the accuracy of the tensor-core Grams' inputs.
// One launch covers K rows k0 .. k0 + Kn - 1 of C (Kn <= 128) and its columns
// c0 .. c0 + Nc - 1; above 128 orbitals the launcher runs blocks of 128 in K and
// in columns, the later K blocks adding into U in float64 (acc).
// ---------------------------------------------------------------------------
constexpr int kRotTcBlk = 128;  // K rows and columns of one launch (exact FP32 level sums, shared memory)

__host__ __device__ constexpr int rot_sbo(int Kp) { return (Kp / 8) * kTcLBO + 16; }

// Threads of a rotation CTA: 256 for Np <= 32 (two CTAs a SM: one converts and
// reads out while the other's MMAs run; 96 TMEM columns each), 512 above.
__host__ __device__ constexpr int rot_threads(int NB) { return NB == 32 ? 256 : 512; }

template <int NB>
__global__ void __launch_bounds__(rot_threads(NB), NB == 32 ? 2 : 1)
    k_rotate_tc(long long G, int N, int Np, int Kp, const float* __restrict__ xh, const double* __restrict__ C,
                double* __restrict__ U, int* __restrict__ status, int k0, int c0, int Nc, int acc) {
  constexpr uint32_t kTmemCols = kTcDigits * NB <= 128 ? 128 : 256;
  constexpr int kThr = rot_threads(NB);
  extern __shared__ __align__(1024) unsigned char smem[];
  const int sbo = rot_sbo(Kp);
  const int aPiece = (kTcM / 8) * sbo;                 // one digit plane of A (128 node rows)
  const int nbp = (Nc + NB - 1) / NB * NB;              // this block's C columns, padded to whole N-tiles
  const int bPiece = (nbp / 8) * sbo;                   // one digit plane of B (all columns)
  unsigned char* aBuf = smem;
  unsigned char* bBuf = smem + kTcDigits * aPiece;
  int* cexpB = reinterpret_cast<int*>(bBuf + kTcDigits * bPiece);  // [nbp] column exponents of C
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ unsigned rmax[kTcM];
  __shared__ int rexp[kTcM];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int koct = Kp / 8;

  // zero the operand planes (K beyond N and columns beyond Nc stay zero)
  const int zbytes = kTcDigits * (aPiece + bPiece);
  for (int i = tid; i < zbytes / 16; i += kThr) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    s_fail = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  // B: the digits of C, row b (column of C), K = a; one exponent per column
  for (int b = tid; b < nbp; b += kThr) {
    unsigned m = 0u;
    if (b < Nc)
      for (int a = 0; a < N; ++a)
        m = max(m, __float_as_uint(__double2float_rn(C[(long long)(k0 + a) * Np + c0 + b])) & 0x7FFFFFFFu);
    cexpB[b] = col_exponent(m);
  }
  __syncthreads();
  for (int w = tid; w < nbp * koct; w += kThr) {
    const int b = w / koct, oct = w % koct;
    const float sc = pow2f(8 - cexpB[b]);
    uint32_t q[kTcDigits][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const int a0 = 8 * oct + j;
      const float cv0 = (b < Nc && a0 < N) ? __double2float_rn(C[(long long)(k0 + a0) * Np + c0 + b]) : 0.f;
      const float cv1 = (b < Nc && a0 + 1 < N) ? __double2float_rn(C[(long long)(k0 + a0 + 1) * Np + c0 + b]) : 0.f;
      float d0[kTcDigits], d1[kTcDigits];
      digits3(cv0, sc, d0);
      digits3(cv1, sc, d1);
#pragma unroll
      for (int p = 0; p < kTcDigits; ++p) q[p][j / 2] = pack_bf16(d0[p], d1[p]);
    }
    unsigned char* dst = bBuf + (uint32_t)((b >> 3) * sbo + oct * kTcLBO + (b & 7) * 16);
#pragma unroll
    for (int p = 0; p < kTcDigits; ++p)
      *reinterpret_cast<uint4*>(dst + p * bPiece) = make_uint4(q[p][0], q[p][1], q[p][2], q[p][3]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  // A conversion items: (node row, octet of a): 128 rows x Kp / 8 octets, at most
  // 4 a thread at 512 threads (Kp <= 128) and 2 at 256 threads (NB = 32: Kp <= 32)
  constexpr int kIt = kTcM * (NB == 32 ? 32 : kRotTcBlk) / 8 / kThr;
  const int nitems = kTcM * koct;
  float v[kIt][8];
  const long long ntiles = (G + kTcM - 1) / kTcM;
  auto load = [&](long long tile) {
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int w = tid + it * kThr;
      const int r = w / koct, oct = w % koct;
      const long long g = tile * kTcM + r;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int a = 8 * oct + j;
        v[it][j] = (w < nitems && tile < ntiles && g < G && a < N) ? __ldg(xh + g * Np + k0 + a) : 0.f;
      }
    }
  };
  const uint32_t idesc = idesc_bf16(kTcM, NB);
  const uint32_t aBase = smem_u32(aBuf), bBase = smem_u32(bBuf);
  const int row = 32 * (warp % 4) + lane;  // node row of this thread in the read-out
  constexpr int kColsT = NB / (kThr / 128);  // columns a thread reads out (4 warps per column group)
  const int col0 = (warp / 4) * kColsT;
  uint32_t phase = 0;
  load(blockIdx.x);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // row maxima -> exponents, then the digits of this tile's X rows
    for (int i = tid; i < kTcM; i += kThr) rmax[i] = 0u;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int w = tid + it * kThr;
      if (w < nitems) {
        unsigned m = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) m = max(m, __float_as_uint(v[it][j]) & 0x7FFFFFFFu);
        if (m) atomicMax(&rmax[w / koct], m);
      }
    }
    __syncthreads();
    for (int i = tid; i < kTcM; i += kThr) rexp[i] = col_exponent(rmax[i]);
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int w = tid + it * kThr;
      if (w < nitems) {
        const int r = w / koct, oct = w % koct;
        const float sc = pow2f(8 - rexp[r]);
        uint32_t q[kTcDigits][4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float d0[kTcDigits], d1[kTcDigits];
          digits3(v[it][j], sc, d0);
          digits3(v[it][j + 1], sc, d1);
#pragma unroll
          for (int p = 0; p < kTcDigits; ++p) q[p][j / 2] = pack_bf16(d0[p], d1[p]);
        }
        unsigned char* dst = aBuf + (uint32_t)((r >> 3) * sbo + oct * kTcLBO + (r & 7) * 16);
#pragma unroll
        for (int p = 0; p < kTcDigits; ++p)
          *reinterpret_cast<uint4*>(dst + p * aPiece) = make_uint4(q[p][0], q[p][1], q[p][2], q[p][3]);
      }
    }
    fence_proxy_async_smem();  // generic writes -> the MMA's async-proxy reads
    load(tile + gridDim.x);    // the next tile's X rows are in flight during the MMAs
    const long long g = tile * kTcM + row;
    const int eg = rexp[row];
    for (int n0 = 0; n0 < Nc; n0 += NB) {
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int l = 0; l < kTcDigits; ++l)
#pragma unroll
          for (int i = 0; i <= l; ++i)
            for (int ks = 0; ks < Kp / 16; ++ks) {
              const uint64_t ad = smem_desc(aBase + i * aPiece + ks * 2 * kTcLBO, kTcLBO, sbo);
              const uint64_t bd =
                  smem_desc(bBase + (l - i) * bPiece + (n0 / 8) * sbo + ks * 2 * kTcLBO, kTcLBO, sbo);
              mma_bf16(tmem + (uint32_t)(l * NB), ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
            }
        mma_commit(&bar);
      }
      bool ok = mbar_wait(&bar, phase);
      if (!ok) {
        s_fail = 1;
        ok = mbar_wait(&bar, phase);  // let the MMAs in flight end before the memory is freed (bounded)
      }
      phase ^= 1;
      tc_fence_after();
      __syncthreads();
      if (s_fail) break;
      // U[g][n0 + b] = 2^(E_g + F_b - 16) (L0 + L1 2^-8 + L2 2^-16), by the warps whose
      // columns include some b < Nc
#pragma unroll
      for (int c = 0; c < kColsT && n0 + col0 < Nc; c += 8) {
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(col0 + c);
        float v0[8], v1[8];
        tmem_ld8(ta, v0);
        tmem_ld8(ta + NB, v1);
        FF tsum[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) two_sum(v0[i], __fmul_rn(v1[i], 0x1p-8f), tsum[i].hi, tsum[i].lo);
        tmem_ld8(ta + 2 * NB, v0);
        double out[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          ff_add(tsum[i], FF{__fmul_rn(v0[i], 0x1p-16f), 0.f});
          const int b = n0 + col0 + c + i;
          // the scale 2^sc on the float pair (exact power-of-two products), then one
          // float64 addition; ldexp in float64 only for scales outside the float range
          const int sc = eg + (b < Nc ? cexpB[b] : 0) - 16;
          const FF tn = ff_norm(tsum[i]);
          if (b >= Nc) out[i] = 0.0;
          else if (sc >= -100 && sc <= 100) out[i] = ff_to_double(FF{__fmul_rn(tn.hi, pow2f(sc)), __fmul_rn(tn.lo, pow2f(sc))});
          else out[i] = ldexp(ff_to_double(tn), sc);
        }
        const int b0 = n0 + col0 + c;
        if (g < G && b0 < Nc) {
          double* dst = U + g * Np + c0 + b0;
#pragma unroll
          for (int i = 0; i < 8; i += 2)
            if (b0 + i < Nc) {
              double2 o = make_double2(out[i], out[i + 1]);
              if (acc) {
                const double2 u = *reinterpret_cast<const double2*>(dst + i);
                o.x += u.x;
                o.y += u.y;
              }
              *reinterpret_cast<double2*>(dst + i) = o;
            }
        }
      }
    }
    if (s_fail) break;
  }
  if (s_fail && tid == 0) atomicOr(status, kStatTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

// One CTA per SM (>= 150 KB of shared memory), chunks a multiple of kTcSuper nodes.
void gram_tc_shape(const Grid& g, long long* chunk, int* nch) {
  const long long want = 152;
  long long ch = (g.G + want - 1) / want;
  ch = (ch + kTcSuper - 1) / kTcSuper * kTcSuper;
  *chunk = ch;
  *nch = (int)((g.G + ch - 1) / ch);
}

size_t gram_tc_partial_doubles(const Grid& g, int Np) {
  long long chunk;
  int nch;
  gram_tc_shape(g, &chunk, &nch);
  return (size_t)nch * Np * Np * (Np <= 32 ? 2 : 1);  // Np <= 32: both Grams' partials
}

// Both Grams of the Rayleigh-Ritz step, G_A = X^T (HX) into partA and G_B =
// X^T (MX) into partB (per-CTA partials [nch][Np][Np] each), in one launch of
// the 64-column kernel with the columns of HX then MX (Np <= 32).
cudaError_t launch_gram_tc_pair(const Grid& g, int Np, const float* xh, const float* ah, const float* bh,
                                double* partA, double* partB, int* n_chunks, int* status, cudaStream_t st) {
  long long chunk;
  int nch;
  gram_tc_shape(g, &chunk, &nch);
  *n_chunks = nch;
  if (Np < 4 || Np % 4 != 0 || Np > 32) return cudaErrorInvalidValue;
  return launch_tc<64>(g.G, Np, 0, Np, 0, 2 * Np, xh, ah, partA, chunk, nch, status, st, bh, Np, partB);
}

// One Gram G = X^T Y into per-CTA partials part[nch][Np][Np] (Np <= kTcMaxNp, a
// multiple of 4; xh, yh 16-byte aligned): blocks of 128 rows x 64 columns (one
// block of 32 columns when Np <= 32).
cudaError_t launch_gram_tc(const Grid& g, int Np, const float* xh, const float* yh, double* part, int* n_chunks,
                           int* status, cudaStream_t st) {
  long long chunk;
  int nch;
  gram_tc_shape(g, &chunk, &nch);
  *n_chunks = nch;
  if (Np < 4 || Np % 4 != 0 || Np > kTcMaxNp) return cudaErrorInvalidValue;
  if (Np <= 32) return launch_tc<32>(g.G, Np, 0, Np, 0, Np, xh, yh, part, chunk, nch, status, st);
  for (int r0 = 0; r0 < Np; r0 += kTcM)
    for (int c0 = 0; c0 < Np; c0 += 64) {
      const int na = Np - r0 < kTcM ? Np - r0 : kTcM, nb = Np - c0 < 64 ? Np - c0 : 64;
      const cudaError_t e = launch_tc<64>(g.G, Np, r0, na, c0, nb, xh, yh, part, chunk, nch, status, st);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace paro

namespace paro {

// U = X C on the tensor cores (Np <= kRotTcMaxNp): X as the float32 hi parts
// [G][Np], C float64 [Np][Np] (zero beyond N), U float64 [G][Np].
cudaError_t launch_rotate_tc(const Grid& g, int N, int Np, const float* xh, const double* C, double* U, int* status,
                             cudaStream_t st) {
  if (Np < 4 || Np % 4 != 0 || Np > kRotTcMaxNp || N > Np) return cudaErrorInvalidValue;
  const long long ntiles = (g.G + kTcM - 1) / kTcM;
  if (Np <= 32) {
    const int Kp = (N + 15) / 16 * 16;
    const int grid = (int)(ntiles < 2 * 152 ? ntiles : 2 * 152);
    const int nbp = 32;
    const size_t smem = (size_t)kTcDigits * ((kTcM / 8) + nbp / 8) * rot_sbo(Kp) + sizeof(int) * nbp;
    cudaError_t e = allow_max_dyn_smem((const void*)k_rotate_tc<32>);
    if (e != cudaSuccess) return e;
    k_rotate_tc<32><<<grid, rot_threads(32), smem, st>>>(g.G, N, Np, Kp, xh, C, U, status, 0, 0, Np, 0);
    return cudaGetLastError();
  }
  // U[:, c0 : c0 + Nc] = sum over K blocks of X[:, k0 : k0 + Kn] C[k0 : k0 + Kn, c0 : c0 + Nc]: blocks of at
  // most 128 in K and in columns, the later K blocks added to U in float64
  const int grid = (int)(ntiles < 152 ? ntiles : 152);
  cudaError_t e = allow_max_dyn_smem((const void*)k_rotate_tc<64>);
  if (e != cudaSuccess) return e;
  for (int c0 = 0; c0 < Np; c0 += kRotTcBlk) {
    const int Nc = Np - c0 < kRotTcBlk ? Np - c0 : kRotTcBlk;
    const int nbp = (Nc + 63) / 64 * 64;
    for (int k0 = 0; k0 < N; k0 += kRotTcBlk) {
      const int Kn = N - k0 < kRotTcBlk ? N - k0 : kRotTcBlk;
      const int Kp = (Kn + 15) / 16 * 16;
      const size_t smem = (size_t)kTcDigits * ((kTcM / 8) + nbp / 8) * rot_sbo(Kp) + sizeof(int) * nbp;
      k_rotate_tc<64><<<grid, rot_threads(64), smem, st>>>(g.G, Kn, Np, Kp, xh, C, U, status, k0, c0, Nc, k0 > 0);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace paro
