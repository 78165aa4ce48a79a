// Batched single-pass Jacobi PCG: the float32 correction solves of Step 3 (the
// shifted source problems A x_i = b_i of eq. 3.2) of many independent systems
// -- uneven meshes, orbital counts and potentials -- in one cooperative launch.
//
// The iteration is that of the single-system kernel (cg2.cu): textbook Jacobi
// PCG with its two reductions merged into one per pass, so pass k forms
// r_k = r_{k-1} - alpha q_{k-1}, z_k = D^-1 r_k, p_k = z_k + beta p_{k-1} at the
// staged neighbours of every node, q_k = A p_k with the 27-point stencil, x_k,
// and the five sums (r,z), (r,r), (p,q), (q,z), (q,D^-1 q); rho_{k+1} follows from
// rho_k - 2 alpha (q,z) + alpha^2 (q,D^-1 q).  Per unit and pass 32 bytes.
//
// What differs is the distribution of the work:
// - work items are (system, orbital block, tile column, z-chunk of zlen planes);
//   each pass every CTA's producer lane takes items from one counter in global
//   memory and stages their planes by TMA (per-system tensor maps in global
//   memory), so the work of systems still iterating spreads over all SMs while
//   converged systems and orbital blocks drop out;
// - the producer hands every staged plane's item to the consumers in a slot
//   header (written before the slot's mbarrier arrival, read after its wait);
// - each consumer warp writes its per-item sums straight to global memory,
//   [item][warp][5][block width]: no CTA barrier among consumers, and the owner
//   CTA of an orbital sums them over the block's items and warps in a fixed
//   order, so results do not depend on which CTA took which item;
// - the owner publishes alpha, beta and the activity of its orbital, and sets
//   its group's bit in the next pass's mask of the orbital block.
// Two bounded grid barriers a pass (partials written / steps published), as in
// the single-system kernel.  Every wait is bounded; a wait that runs out sets
// the timeout bit of every system in the launch and the kernel returns.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "cg.cuh"
#include "cgutil.cuh"
#include "cg2util.cuh"
#include "tma.cuh"

namespace paro {

namespace {

// Slot header: the item a staged plane belongs to, written by the producer lane
// before the slot's arrival.  The write pointers of the item's system sit here
// too, so the consumers keep them out of registers.
struct SlotHdr {
  int item, s, z0, z1, x0, y0, sys, na;
  int list[8];  // the item's active groups (global group index in the system)
  float *wx, *wr, *wq, *wp;
  long long plane4;  // floats per z plane of one group
};
constexpr int kMaxJobsB = 4096;  // orbital blocks of one batch (their masks sit in shared memory)

__device__ __forceinline__ bool in_mask(const unsigned long long* m, int s) { return (m[s >> 6] >> (s & 63)) & 1ull; }

// Orbital o of system s takes part in the first pass.
__device__ __forceinline__ bool act0(const CG2BArgs& a, const CG2BSys& sy, int s, int o) {
  return in_mask(a.part_mask, s) && o < sy.N && sy.st->maxit > 0 && sy.st->skip[o] == 0;
}

template <int G4, int NPT>
__global__ void __launch_bounds__(cg2_max_threads(NPT), 1) k_cg2b(CG2BArgs a, K1Geom geo) {
  constexpr int bw = 4 * G4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int TX = geo.TX, TY = geo.TY;
  const int HX = TX + 2, HY = TY + 2;
  const int nthr = geo.nthr;
  const int NC = nthr * G4;
  const int S = geo.slots;
  const int tid = threadIdx.x;
  const bool producer = tid >= NC;
  const int j = tid % nthr;
  const int k = tid / nthr;
  const int lane = tid & 31;
  const int vecf = HY * HX * 4;
  const int vstr = box_stride_floats(HX, HY);
  const unsigned spin = a.spin;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxSlots2;
  unsigned char* base = smem + 128;
  auto slotR = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes); };
  auto slotQ = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_p); };
  auto slotP = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_s); };
  auto slotD = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_d); };
  auto slotW = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_w); };
  unsigned* smask = reinterpret_cast<unsigned*>(base + (size_t)S * geo.slot_bytes);  // [njobs] this pass
  __shared__ SlotHdr s_hdr[kMaxSlots2];
  __shared__ int s_any, s_gok, s_lstep;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC / 32);
    }
    fence_mbar_init();
  }
  // the systems' open counts are summed by the owners at the end (after at least
  // one pair of grid barriers when any orbital iterates)
  if (blockIdx.x == 0)
    for (int s = tid; s < a.nsys; s += blockDim.x)
      if (in_mask(a.part_mask, s)) a.sys[s].st->n_active = 0;
  __syncthreads();

  const uint32_t vbytes = (uint32_t)vecf * 4u;
  const uint32_t dwbytes = (uint32_t)(geo.DX * HY + kW2 * TX * TY) * 4u;
  const unsigned long long per_pass = (unsigned long long)a.nitems + gridDim.x;
  unsigned long long ibase = 0;  // the item counter's value at the start of this pass
  bool first = true;
  int rd = 0;
  int lstep = 0, cstep = 0;
  bool timed_out = false;
  int npass = 0;
  if (tid == 0) s_lstep = 0;

  // producer (one lane): items from the counter until it runs past the pass's
  // items, every staged plane announced in its slot header; then an end marker
  auto produce = [&]() -> bool {
    for (;;) {
      const unsigned long long t = atomicAdd(a.ictr, 1ull);
      const long long idx = (long long)(t - ibase);
      const bool end = idx >= a.nitems;
      int4 it = make_int4(0, 0, 0, 0);
      unsigned mask = 0u;
      if (!end) {
        it = __ldg(&a.items[idx]);
        mask = smask[it.x];
        if (mask == 0u) continue;
      }
      if (end) {
        const int slot = lstep % S;
        if (lstep >= S && !mbar_wait_n(&empty[slot], ((lstep / S) - 1) & 1, spin)) return false;
        s_hdr[slot].item = -1;
        mbar_arrive(&full[slot]);
        ++lstep;
        return true;
      }
      const CG2BJob J = a.jobs[it.x];
      const int sy = J.sys;
      const CG2BSys& Sy = a.sys[sy];
      const int nz = Sy.g.nz;
      const int x0 = 1 + it.y * TX, y0 = 1 + it.z * TY;
      const int z0 = 1 + it.w * a.zlen;
      const int z1 = min(z0 + a.zlen, nz);
      const int na = __popc(mask);
      const CUtensorMap* M = a.maps + (size_t)sy * 8;
      const CUtensorMap* R = M + (rd ? 3 : 0);
      const CUtensorMap* Q = M + (rd ? 4 : 1);
      const CUtensorMap* P = M + (rd ? 5 : 2);
      for (int zin = z0 - 1; zin <= z1; ++zin) {
        const int slot = lstep % S;
        if (lstep >= S && !mbar_wait_n(&empty[slot], ((lstep / S) - 1) & 1, spin)) return false;
        SlotHdr* h = &s_hdr[slot];
        h->item = (int)idx;
        h->s = zin;
        h->z0 = z0;
        h->z1 = z1;
        h->x0 = x0;
        h->y0 = y0;
        h->sys = sy;
        h->na = na;
        h->wx = Sy.x;
        h->wr = Sy.r[rd ^ 1];
        h->wq = Sy.q[rd ^ 1];
        h->wp = Sy.p[rd ^ 1];
        h->plane4 = 4ll * Sy.g.Px * Sy.g.Py;
        unsigned mm = mask;
        for (int kk = 0; mm; ++kk) {
          h->list[kk] = J.ob * G4 + __ffs(mm) - 1;  // the kk-th active group of the block
          mm &= mm - 1;
        }
        // the header's writes before the arrival (release): the consumers read it
        // after their wait on this phase (acquire)
        mbar_arrive_expect_tx(&full[slot], (uint32_t)na * (first ? 1u : 3u) * vbytes + dwbytes);
        unsigned mm2 = mask;
        for (int kk = 0; mm2; ++kk) {
          const int gam = J.ob * G4 + __ffs(mm2) - 1;
          mm2 &= mm2 - 1;
          tma_load_4d(slotR(slot) + kk * vstr, R, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
          if (!first) {
            tma_load_4d(slotQ(slot) + kk * vstr, Q, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
            tma_load_4d(slotP(slot) + kk * vstr, P, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
          }
        }
        tma_load_3d(slotD(slot), M + 6, x0 - 1, y0 - 1, zin, &full[slot]);
        tma_load_4d(slotW(slot), M + 7, 0, x0 - 1, y0 - 1, zin, &full[slot]);
        ++lstep;
      }
    }
  };

  const int tx = j % TX, ty0 = (j / TX) * NPT;
  const int wpg = nthr >> 5;           // warps of one group slot
  const int wslot = (tid >> 5) % wpg;  // this warp within its group slot

  // consumers: the staged planes in ring order until the end marker; false on a
  // timed-out wait (no consumer barrier: the other warps and the producer time
  // out on their own bounded waits)
  auto consume = [&]() -> bool {
    float dt[kDots][4];
    bool kact = false;
    float al[4], be[4];
    bool inside[NPT];
    long long ebase[NPT];  // float offset of own node i in plane 0 of this thread's group
    Vec4<float> aU[NPT], aC[NPT], aD[NPT], pv_z[NPT], pv_p[NPT], xnext[NPT];
    float pv_d[NPT];
    const int DX = geo.DX;
    for (;;) {
      const int slot = cstep % S;
      const uint32_t par = (cstep / S) & 1;
      if (!mbar_wait_n(&full[slot], par, spin)) return false;
      const SlotHdr* h = &s_hdr[slot];
      if (h->item < 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        ++cstep;
        return true;
      }
      const int s = h->s;
      const int z0 = h->z0, z1 = h->z1;
      if (s == z0 - 1) {
        // first staged plane of an item: its system, tile and active groups
        kact = k < h->na;
        const int gam = kact ? h->list[k] : 0;
        const CG2BSys& Sy = a.sys[h->sys];
        const int Px = Sy.g.Px;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int go = Sy.o0 + 4 * gam + c;
          al[c] = (kact && !first) ? __ldcg(a.oal + go) : 0.f;
          be[c] = (kact && !first) ? __ldcg(a.obe + go) : 0.f;
        }
        const int xg = h->x0 + tx;
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          const int yg = h->y0 + ty0 + i;
          inside[i] = xg <= Sy.g.nx - 1 && yg <= Sy.g.ny - 1;
          ebase[i] = ((long long)gam * Sy.g.G + (long long)yg * Px + xg) * 4;
          aU[i] = aC[i] = aD[i] = pv_z[i] = pv_p[i] = xnext[i] = Vec4<float>{};
          pv_d[i] = 0.f;
        }
#pragma unroll
        for (int d = 0; d < kDots; ++d)
#pragma unroll
          for (int c = 0; c < 4; ++c) dt[d][c] = 0.f;
      }
      const long long plane4 = h->plane4;
      float* const wx = h->wx;
      const bool zout = s >= z0 && s < z1;
      long long eown[NPT];
      Vec4<float> xv[NPT];
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        eown[i] = ebase[i] + (long long)s * plane4;
        xv[i] = xnext[i];
        if (!first && kact && inside[i] && s + 1 >= z0 && s + 1 < z1) xnext[i] = ldcg4(wx + eown[i] + plane4);
      }
      // the item's partial-sum row and this thread's group, read while the slot is held
      const int item = h->item;
      const int gl = kact ? h->list[k] % G4 : 0;  // group within its orbital block
      Vec4<float> cz[NPT], cp[NPT];
      float cd[NPT];
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        cz[i] = cp[i] = Vec4<float>{};
        cd[i] = 0.f;
      }
      if (kact) {
        const float* R = slotR(slot) + k * vstr;
        const float* Q = slotQ(slot) + k * vstr;
        const float* P = slotP(slot) + k * vstr;
        const float* D = slotD(slot);
        Vec4<float> w[NPT][7];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          const float* Wn = slotW(slot) + ((ty0 + i) * TX + tx) * kW2;
#pragma unroll
          for (int q = 0; q < 7; ++q) w[i][q] = lds4(Wn + 4 * q);
        }
#pragma unroll
        for (int cy = 0; cy < NPT + 2; ++cy) {
#pragma unroll
          for (int cxi = 0; cxi < 3; ++cxi) {
            const int hnode = (ty0 + cy) * HX + (tx + cxi);
            const int e = hnode * 4;
            const float d = D[(ty0 + cy) * DX + tx + cxi];
            const Vec4<float> rv = lds4(R + e);
            Vec4<float> qv{}, pv{};
            if (!first) {
              qv = lds4(Q + e);
              pv = lds4(P + e);
            }
            Vec4<float> rn, zn, pn;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              rn.v[c] = fmaf(-al[c], qv.v[c], rv.v[c]);
              zn.v[c] = d * rn.v[c];
              pn.v[c] = fmaf(be[c], pv.v[c], zn.v[c]);
            }
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
              const int cyr = cy - i;
              if (cyr < 0 || cyr > 2) continue;
              const int o = cyr * 3 + cxi;
              const float wu = w[i][o / 4].v[o % 4];
              const float wc = w[i][(9 + o) / 4].v[(9 + o) % 4];
              const float wd = w[i][(18 + o) / 4].v[(18 + o) % 4];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                aU[i].v[c] = fmaf(wu, pn.v[c], aU[i].v[c]);
                aC[i].v[c] = fmaf(wc, pn.v[c], aC[i].v[c]);
                aD[i].v[c] = fmaf(wd, pn.v[c], aD[i].v[c]);
              }
              if (cyr == 1 && cxi == 1) {
                cd[i] = d;
                cz[i] = zn;
                cp[i] = pn;
                if (zout && inside[i]) {
                  Vec4<float> xn;
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    xn.v[c] = fmaf(al[c], pv.v[c], xv[i].v[c]);
                    dt[0][c] = fmaf(rn.v[c], zn.v[c], dt[0][c]);
                    dt[1][c] = fmaf(rn.v[c], rn.v[c], dt[1][c]);
                  }
                  sts4(h->wr + eown[i], rn);
                  sts4(h->wp + eown[i], pn);
                  sts4(wx + eown[i], xn);
                }
              }
            }
          }
        }
      }
      float* const wq = h->wq;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (kact) {
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          const bool prev_out = inside[i] && s - 1 >= z0 && s - 1 < z1;
          if (prev_out) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              dt[2][c] = fmaf(pv_p[i].v[c], aD[i].v[c], dt[2][c]);
              dt[3][c] = fmaf(aD[i].v[c], pv_z[i].v[c], dt[3][c]);
              dt[4][c] = fmaf(aD[i].v[c], pv_d[i] * aD[i].v[c], dt[4][c]);
            }
            sts4(wq + eown[i] - plane4, aD[i]);
          }
          aD[i] = aC[i];
          aC[i] = aU[i];
          aU[i] = Vec4<float>{};
        }
      }
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        pv_z[i] = cz[i];
        pv_p[i] = cp[i];
        pv_d[i] = cd[i];
      }
      ++cstep;
      if (s == z1 && kact) {
        // the item is complete: this warp's sums over its 32 node slots, written
        // to the item's partials (the warp's own row: no barrier)
#pragma unroll
        for (int d = 0; d < kDots; ++d)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float v = dt[d][c];
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
            dt[d][c] = v;
          }
        if (lane < kDots * 4) {
          const int d = lane >> 2, c = lane & 3;
          float v = 0.f;
#pragma unroll
          for (int dd = 0; dd < kDots; ++dd)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
              if (dd == d && cc == c) v = dt[dd][cc];
          a.part[(((long long)item * wpg + wslot) * kDots + d) * bw + 4 * gl + c] = (double)v;
        }
      }
    }
  };

  // bounded grid barrier: arrival `target` of the launch's counter
  auto grid_sync = [&](unsigned target) -> bool {
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      atomicAdd(a.bar, 1u);
      int okb = 0;
      for (unsigned i = 0; i < spin; ++i) {
        if (ld_acquire_u32(a.bar) >= target) {
          okb = 1;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
      s_gok = okb;
    }
    __syncthreads();
    return s_gok != 0;
  };

  const int nwarp = blockDim.x >> 5;
  const int warp = tid >> 5;
  for (npass = 0;; ++npass) {
    // the orbital blocks' active groups for this pass
    if (npass == 0) {
      for (int jb = tid; jb < a.njobs; jb += blockDim.x) {
        const CG2BJob J = a.jobs[jb];
        const CG2BSys& Sy = a.sys[J.sys];
        unsigned m = 0u;
        for (int g = 0; g < J.ng; ++g)
          for (int c = 0; c < 4; ++c)
            if (act0(a, Sy, J.sys, J.ob * bw + 4 * g + c)) m |= 1u << g;
        smask[jb] = m;
      }
    } else {
      for (int jb = tid; jb < a.njobs; jb += blockDim.x) smask[jb] = __ldcg(a.jmask + (size_t)(npass & 1) * a.njobs + jb);
    }
    if (tid == 0) s_any = 0;
    __syncthreads();
    for (int jb = tid; jb < a.njobs; jb += blockDim.x)
      if (smask[jb]) s_any = 1;
    __syncthreads();
    if (!s_any) break;
    if (blockIdx.x == 0) {
      // the next pass's masks (read in the previous pass, set by this pass's owners
      // after the first barrier) and the work counters of the systems
      for (int jb = tid; jb < a.njobs; jb += blockDim.x) {
        a.jmask[(size_t)((npass + 1) & 1) * a.njobs + jb] = 0u;
        const unsigned m = smask[jb];
        if (m) {
          const CG2BSys& Sy = a.sys[a.jobs[jb].sys];
          atomicAdd(&Sy.st->work, 4ull * (unsigned long long)__popc(m) * (unsigned long long)Sy.g.nI);
          atomicAdd(&Sy.st->work_nodes, (unsigned long long)Sy.g.nI);
        }
      }
    }
    __syncthreads();
    bool ok = true;
    if (producer) {
      if (tid == NC) {
        fence_proxy_async_global2();  // the previous pass's generic stores before this pass's TMA reads
        ok = produce();
      }
      __syncwarp();
    } else {
      ok = consume();
    }
    if (tid == NC) s_lstep = lstep;
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    first = false;
    rd ^= 1;
    ibase += per_pass;
    fence_proxy_async_global2();
    if (!grid_sync((2u * npass + 1u) * gridDim.x)) {
      timed_out = true;
      break;
    }
    // owners: a warp per orbital (o mod grid), its five sums over the block's items
    // and warps in a fixed order, the scalar step, published
    for (int go = blockIdx.x + warp * gridDim.x; go < a.norb; go += nwarp * gridDim.x) {
      const int s = a.osys[go];
      const CG2BSys& Sy = a.sys[s];
      const int o = go - Sy.o0;
      const bool act = npass == 0 ? act0(a, Sy, s, o) : __ldcg(a.oact + go) != 0;
      if (!act) {
        if (npass == 0 && lane == 0) {
          a.oact[go] = 0;
          a.oal[go] = 0.f;
          a.obe[go] = 0.f;
          a.oit[go] = 0;
          a.obb[go] = 0.0;
        }
        continue;
      }
      const CG2BJob J = a.jobs[Sy.job0 + o / bw];
      const int gl = o - (o / bw) * bw;
      const int nrow = J.nit * a.wpg;
      double v[kDots];
#pragma unroll
      for (int d = 0; d < kDots; ++d) v[d] = 0.0;
      for (int rrow = lane; rrow < nrow; rrow += 32) {
        const double* src = a.part + ((long long)J.it0 * a.wpg + rrow) * kDots * bw + gl;
#pragma unroll
        for (int d = 0; d < kDots; ++d) v[d] += __ldcg(src + d * bw);
      }
#pragma unroll
      for (int d = 0; d < kDots; ++d)
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v[d] += __shfl_xor_sync(0xffffffffu, v[d], m);
      if (lane == 0) {
        const double rho = v[0], rr = v[1], pq = v[2], qz = v[3], qdq = v[4];
        int status = 0;
        bool still = true;
        double alpha = 0.0, beta = 0.0;
        int it = 0;
        if (npass == 0) {
          a.obb[go] = rr;  // r_0 = b
        } else {
          it = a.oit[go] + 1;  // x was updated in this pass
          Sy.st->rr[o] = rr;
        }
        a.oit[go] = it;
        const double bb = npass == 0 ? rr : a.obb[go];
        const double tol = Sy.st->tol;
        if (!(isfinite(rho) && isfinite(rr) && isfinite(pq) && isfinite(qz) && isfinite(qdq))) {
          status |= kStatNonFinite;
          still = false;
        } else if (npass > 0 && rr <= tol * tol * bb) {
          still = false;
        } else if (npass > 0 && it >= Sy.st->maxit) {
          if (!a.inner) status |= kStatNotConverged;
          still = false;
        }
        if (still) {
          if (!(rho > 0.0) || !(pq > 0.0)) {
            status |= kStatNotSPD;
            still = false;
          } else {
            alpha = rho / pq;
            const double rho1 = rho - 2.0 * alpha * qz + alpha * alpha * qdq;
            beta = rho1 > 0.0 ? rho1 / rho : 0.0;
          }
        }
        atomicAdd(&Sy.st->work_act, (unsigned long long)Sy.g.nI);
        a.oal[go] = still ? (float)alpha : 0.f;
        a.obe[go] = still ? (float)beta : 0.f;
        a.oact[go] = still ? 1 : 0;
        if (still) atomicOr(a.jmask + (size_t)((npass + 1) & 1) * a.njobs + Sy.job0 + o / bw, 1u << (gl >> 2));
        if (status) atomicOr(&Sy.st->status, status);
      }
    }
    if (!grid_sync((2u * npass + 2u) * gridDim.x)) {
      timed_out = true;
      break;
    }
  }
  if (timed_out) {
    if (tid == 0) {
      for (int s = 0; s < a.nsys; ++s)
        if (in_mask(a.part_mask, s)) atomicOr(&a.sys[s].st->status, kStatTimeout);
      for (int q = cstep; q < s_lstep; ++q) mbar_wait_n(&full[q % S], (q / S) & 1, kSpinLimit);
    }
    __syncthreads();
    return;
  }
  // the owners: per-orbital results of the systems in the launch
  for (int go = blockIdx.x + warp * gridDim.x; go < a.norb; go += nwarp * gridDim.x) {
    if (lane != 0) continue;
    const int s = a.osys[go];
    if (!in_mask(a.part_mask, s)) continue;
    const CG2BSys& Sy = a.sys[s];
    const int o = go - Sy.o0;
    const bool ran = npass > 0;
    const int it = ran ? a.oit[go] : 0;
    const int act = ran ? a.oact[go] : 0;
    Sy.st->iters[o] = it;
    Sy.st->bb[o] = ran ? a.obb[go] : 0.0;
    Sy.st->active[o] = act;
    if (act) atomicAdd(&Sy.st->n_active, 1);
    if (it) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&Sy.st->it_sum), (unsigned long long)it);
      atomicMax(&Sy.st->it_max, it);
    }
  }
}

template <int NPT>
void* cg2b_fn_npt(int G4) {
  switch (G4) {
    case 1: return (void*)k_cg2b<1, NPT>;
    case 2: return (void*)k_cg2b<2, NPT>;
    case 3: return (void*)k_cg2b<3, NPT>;
    case 4: return (void*)k_cg2b<4, NPT>;
    case 5: return (void*)k_cg2b<5, NPT>;
    case 6: return (void*)k_cg2b<6, NPT>;
    case 7: return (void*)k_cg2b<7, NPT>;
    case 8: return (void*)k_cg2b<8, NPT>;
  }
  return nullptr;
}

void* cg2b_fn(int G4, int npt) { return npt == 2 ? cg2b_fn_npt<2>(G4) : npt == 1 ? cg2b_fn_npt<1>(G4) : nullptr; }

__global__ void k_fill_interior_gm_b(Grid g, int Np, float* b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * Np) return;
  const int o = (int)(t % Np);
  const long long gp = interior_to_padded(g, (int)(t / Np));
  b[((long long)(o / 4) * g.G + gp) * 4 + o % 4] = 1.0f;
}

}  // namespace

// Shared memory of one CTA: the ring of slots as in the single-system kernel
// (r, q, p boxes of G4 groups, D^-1 and the packed weights of a plane) and the
// orbital blocks' masks of the pass.
static bool cg2b_layout(int bw, int TX, int TY, int npt, int njobs, size_t limit, K1Geom* G) {
  const size_t sz = sizeof(float);
  const int G4 = bw / 4;
  G->TX = TX;
  G->TY = TY;
  G->npt = npt;
  G->nthr = TX * TY / npt;
  G->G4 = G4;
  const int HX = TX + 2, HY = TY + 2;
  G->DX = TX + 4;
  const size_t vec = (size_t)G4 * box_stride_floats(HX, HY) * sz;
  const size_t dv = (size_t)G->DX * HY * sz;
  const size_t wv = (size_t)kW2 * TX * TY * sz;
  auto al = [](size_t v) { return (v + 127) / 128 * 128; };
  G->off_p = (int)al(vec);
  G->off_s = (int)(G->off_p + al(vec));
  G->off_d = (int)(G->off_s + al(vec));
  G->off_w = (int)(G->off_d + al(dv));
  G->slot_bytes = (int)(G->off_w + al(wv));
  G->tx_bytes = (uint32_t)(3 * (size_t)G4 * HX * HY * 16 + dv + wv);
  const size_t red = (size_t)njobs * 4 + 16;
  if (128 + red + 3 * (size_t)G->slot_bytes > limit) return false;
  int slots = (int)((limit - 128 - red) / G->slot_bytes);
  if (slots > kMaxSlots2) slots = kMaxSlots2;
  G->slots = slots;
  G->smem = 128 + (size_t)slots * G->slot_bytes + red;
  return true;
}

void cg2b_candidates(const CG2BPlan* P, std::vector<K1Geom>* out) {
  out->clear();
  int npmax = 4;
  for (const auto& d : P->desc) npmax = d.Np > npmax ? d.Np : npmax;
  const size_t stat = sizeof(SlotHdr) * kMaxSlots2 + 64;
  const size_t limit = 227 * 1024 - stat - 1024;
  // the two-node slot shapes first (the single-system kernel's best), then one node a thread
  const int shapes[8][3] = {{32, 4, 2}, {16, 8, 2}, {8, 16, 2}, {16, 4, 1}, {8, 8, 1}, {16, 6, 1}, {24, 4, 1}, {8, 12, 1}};
  const int g4s[6] = {4, 2, 3, 5, 6, 8};
  for (int gi = 0; gi < 6; ++gi) {
    const int G4 = g4s[gi];
    if (4 * G4 > ((npmax + 3) / 4) * 4 && G4 > 1) continue;  // wider than the widest system
    for (int si = 0; si < 8; ++si) {
      const int TX = shapes[si][0], TY = shapes[si][1], npt = shapes[si][2];
      if (TX * TY / npt * G4 + 32 > cg2_max_threads(npt)) continue;
      int njobs = 0;
      for (const auto& d : P->desc) njobs += (d.Np + 4 * G4 - 1) / (4 * G4);
      if (njobs > kMaxJobsB) continue;
      K1Geom G{};
      if (!cg2b_layout(4 * G4, TX, TY, npt, njobs, limit, &G)) continue;
      G.nob = njobs;
      out->push_back(G);
    }
  }
}

static cudaError_t cg2b_alloc_bytes(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  return e;
}

cudaError_t cg2b_create(CG2BPlan* P, const std::vector<CG2BSysDesc>& sys, int nsm) {
  if (sys.empty() || sys.size() > (size_t)kMaxBatchSys) return cudaErrorInvalidValue;
  P->desc = sys;
  P->nsm = nsm;
  int norb = 0;
  for (const auto& d : sys) {
    if (d.Np % 4 || d.Np < 4 || d.N < 1 || d.N > d.Np) return cudaErrorInvalidValue;
    norb += d.Np;
  }
  cudaError_t e;
  if ((e = cg2b_alloc_bytes((void**)&P->dsys, sizeof(CG2BSys) * sys.size())) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->dmaps, sizeof(CUtensorMap) * 8 * sys.size())) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->dosys, sizeof(int) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->dobb, sizeof(double) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->doit, sizeof(int) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->doact, sizeof(int) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->doal, sizeof(float) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->dobe, sizeof(float) * norb)) != cudaSuccess) return e;
  if ((e = cg2b_alloc_bytes((void**)&P->dbar, 64)) != cudaSuccess) return e;
  std::vector<int> osys(norb);
  for (int s = 0, o = 0; s < (int)sys.size(); ++s)
    for (int i = 0; i < sys[s].Np; ++i) osys[o++] = s;
  if ((e = cudaMemcpy(P->dosys, osys.data(), sizeof(int) * norb, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  CG2BArgs& a = P->args;
  a.nsys = (int)sys.size();
  a.norb = norb;
  a.osys = P->dosys;
  a.obb = P->dobb;
  a.oit = P->doit;
  a.oact = P->doact;
  a.oal = P->doal;
  a.obe = P->dobe;
  a.bar = P->dbar;
  a.ictr = reinterpret_cast<unsigned long long*>(P->dbar + 8);
  a.spin = kSpinLimit;
  a.inner = 1;
  std::vector<K1Geom> cand;
  cg2b_candidates(P, &cand);
  if (cand.empty()) return cudaErrorInvalidConfiguration;
  return cg2b_prepare_geo(P, cand[0]);
}

void cg2b_destroy(CG2BPlan* P) {
  void* ps[] = {P->dsys, P->djobs, P->ditems, P->dmaps, P->dosys, P->dpart, P->dobb,
                P->doit, P->doact, P->doal, P->dobe, P->djmask, P->dbar};
  for (void* p : ps)
    if (p) cudaFree(p);
}

// Work tables of a geometry (host only): the orbital blocks (jobs) of every
// system in order and their items (tile column x z-chunk), with whole columns
// unless that gives fewer than 8 items a CTA (then chunks of at least 16 planes).
void cg2b_tables(const std::vector<CG2BSysDesc>& desc, const K1Geom& G, std::vector<CG2BJob>* jobs,
                 std::vector<int4>* items, int* zlen_out) {
  const int G4 = G.G4, bw = 4 * G4;
  int nzmax = 1;
  for (const auto& d : desc) nzmax = d.g.nz - 1 > nzmax ? d.g.nz - 1 : nzmax;
  auto count_items = [&](int zl) {
    long long n = 0;
    for (const auto& d : desc) {
      const int ncx = (d.g.nx - 1 + G.TX - 1) / G.TX, ncy = (d.g.ny - 1 + G.TY - 1) / G.TY;
      n += (long long)((d.Np + bw - 1) / bw) * ncx * ncy * ((d.g.nz - 1 + zl - 1) / zl);
    }
    return n;
  };
  int zlen = nzmax;
  while (zlen > 16 && count_items(zlen) < 8LL * G.grid) zlen = (zlen + 1) / 2;
  *zlen_out = zlen;
  jobs->clear();
  items->clear();
  for (int s = 0; s < (int)desc.size(); ++s) {
    const CG2BSysDesc& d = desc[s];
    const int ncx = (d.g.nx - 1 + G.TX - 1) / G.TX, ncy = (d.g.ny - 1 + G.TY - 1) / G.TY;
    const int nob = (d.Np + bw - 1) / bw;
    const int nzc = (d.g.nz - 1 + zlen - 1) / zlen;
    for (int ob = 0; ob < nob; ++ob) {
      CG2BJob J{};
      J.sys = s;
      J.ob = ob;
      J.ng = (d.Np / 4 - ob * G4) < G4 ? d.Np / 4 - ob * G4 : G4;
      J.it0 = (int)items->size();
      for (int ty = 0; ty < ncy; ++ty)
        for (int tx = 0; tx < ncx; ++tx)
          for (int zc = 0; zc < nzc; ++zc) items->push_back(make_int4((int)jobs->size(), tx, ty, zc));
      J.nit = (int)items->size() - J.it0;
      jobs->push_back(J);
    }
  }
}

// Geometry: jobs (orbital blocks) and items (tile columns in z-chunks) of every
// system, the systems' tensor maps for the tile, kernel attributes and the
// co-residency check of the cooperative grid.
cudaError_t cg2b_prepare_geo(CG2BPlan* P, const K1Geom& geo) {
  P->ok = false;
  P->geo = geo;
  K1Geom& G = P->geo;
  CG2BArgs& a = P->args;
  const int G4 = G.G4, bw = 4 * G4;
  const int nsys = (int)P->desc.size();
  // grid: one CTA per SM (all co-resident)
  G.grid = P->nsm < kMaxGrid1 ? P->nsm : kMaxGrid1;
  std::vector<CG2BJob> jobs;
  std::vector<int4> items;
  cg2b_tables(P->desc, G, &jobs, &items, &a.zlen);
  P->hsys.assign(nsys, CG2BSys{});
  for (int s = 0, o0 = 0; s < nsys; ++s) {
    const CG2BSysDesc& d = P->desc[s];
    CG2BSys& Y = P->hsys[s];
    Y.g = d.g;
    Y.Np = d.Np;
    Y.N = d.N;
    Y.ncx = (d.g.nx - 1 + G.TX - 1) / G.TX;
    Y.ncy = (d.g.ny - 1 + G.TY - 1) / G.TY;
    Y.o0 = o0;
    Y.job0 = 0;
    while (Y.job0 < (int)jobs.size() && jobs[Y.job0].sys != s) ++Y.job0;
    Y.x = d.x;
    for (int b = 0; b < 2; ++b) {
      Y.r[b] = d.r[b];
      Y.q[b] = d.q[b];
      Y.p[b] = d.p[b];
    }
    Y.st = d.st;
    o0 += d.Np;
  }
  if ((int)jobs.size() > kMaxJobsB) return cudaErrorInvalidConfiguration;
  G.nob = (int)jobs.size();
  a.njobs = (int)jobs.size();
  a.nitems = (int)items.size();
  a.wpg = G.nthr / 32;
  cudaError_t e;
  if (jobs.size() > P->jobs_cap) {
    if (P->djobs) cudaFree(P->djobs);
    if (P->djmask) cudaFree(P->djmask);
    P->djobs = nullptr;
    P->djmask = nullptr;
    if ((e = cg2b_alloc_bytes((void**)&P->djobs, sizeof(CG2BJob) * jobs.size())) != cudaSuccess) return e;
    if ((e = cg2b_alloc_bytes((void**)&P->djmask, sizeof(unsigned) * 2 * jobs.size())) != cudaSuccess) return e;
    P->jobs_cap = jobs.size();
  }
  if (items.size() > P->items_cap) {
    if (P->ditems) cudaFree(P->ditems);
    P->ditems = nullptr;
    if ((e = cg2b_alloc_bytes((void**)&P->ditems, sizeof(int4) * items.size())) != cudaSuccess) return e;
    P->items_cap = items.size();
  }
  const size_t npart = items.size() * (size_t)a.wpg * kDots * bw;
  if (npart > P->part_cap) {
    if (P->dpart) cudaFree(P->dpart);
    P->dpart = nullptr;
    if ((e = cg2b_alloc_bytes((void**)&P->dpart, sizeof(double) * npart)) != cudaSuccess) return e;
    P->part_cap = npart;
  }
  if ((e = cudaMemcpy(P->djobs, jobs.data(), sizeof(CG2BJob) * jobs.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpy(P->ditems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpy(P->dsys, P->hsys.data(), sizeof(CG2BSys) * nsys, cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  // tensor maps of every system for this tile: the single-system kernel's boxes
  std::vector<CUtensorMap> maps((size_t)nsys * 8);
  const uint64_t sz = sizeof(float);
  const CUtensorMapDataType ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (int s = 0; s < nsys; ++s) {
    const CG2BSysDesc& d = P->desc[s];
    CUtensorMap* M = &maps[(size_t)s * 8];
    uint64_t dims[4] = {(uint64_t)4 * d.g.Px, (uint64_t)d.g.Py, (uint64_t)d.g.Pz, (uint64_t)(d.Np / 4)};
    uint64_t str[3] = {(uint64_t)4 * d.g.Px * sz, (uint64_t)4 * d.g.Px * d.g.Py * sz, (uint64_t)4 * d.g.G * sz};
    uint32_t box[4] = {(uint32_t)(4 * (G.TX + 2)), (uint32_t)(G.TY + 2), 1, 1};
    for (int b = 0; b < 2; ++b) {
      if ((e = encode_tiled(&M[3 * b + 0], ty, 4, d.r[b], dims, str, box)) != cudaSuccess) return e;
      if ((e = encode_tiled(&M[3 * b + 1], ty, 4, d.q[b], dims, str, box)) != cudaSuccess) return e;
      if ((e = encode_tiled(&M[3 * b + 2], ty, 4, d.p[b], dims, str, box)) != cudaSuccess) return e;
    }
    uint64_t ddims[3] = {(uint64_t)d.dpitch, (uint64_t)d.g.Py, (uint64_t)d.g.Pz};
    uint64_t dstr[2] = {(uint64_t)d.dpitch * sz, (uint64_t)d.dpitch * d.g.Py * sz};
    uint32_t dbox[3] = {(uint32_t)G.DX, (uint32_t)(G.TY + 2), 1};
    if ((e = encode_tiled(&M[6], ty, 3, (void*)d.dinv_tma, ddims, dstr, dbox)) != cudaSuccess) return e;
    const uint64_t nxi = (uint64_t)(d.g.nx - 1), nyi = (uint64_t)(d.g.ny - 1);
    uint64_t wdims[4] = {(uint64_t)kW2, nxi, nyi, (uint64_t)d.g.Pz};
    uint64_t wstr[3] = {(uint64_t)kW2 * sz, (uint64_t)kW2 * nxi * sz, (uint64_t)kW2 * nxi * nyi * sz};
    uint32_t wbox[4] = {(uint32_t)kW2, (uint32_t)G.TX, (uint32_t)G.TY, 1};
    if ((e = encode_tiled(&M[7], ty, 4, (void*)d.wcoef, wdims, wstr, wbox)) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpy(P->dmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  a.sys = P->dsys;
  a.jobs = P->djobs;
  a.items = P->ditems;
  a.maps = P->dmaps;
  a.part = P->dpart;
  a.jmask = P->djmask;
  void* f = cg2b_fn(G4, G.npt);
  if (!f) return cudaErrorInvalidValue;
  if ((e = allow_max_dyn_smem(f)) != cudaSuccess) return e;
  int nb = 0, dev = 0, coop = 0;
  P->ok = cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, G.nthr * G4 + 32, G.smem) == cudaSuccess &&
          (long long)nb * P->nsm >= G.grid;
  (void)cudaGetLastError();
  return cudaSuccess;
}

cudaError_t cg2b_launch(CG2BPlan* P, const unsigned long long* mask, unsigned spin, cudaStream_t st) {
  if (!P->ok) return cudaErrorInvalidConfiguration;
  CG2BArgs a = P->args;
  for (int i = 0; i < kMaxBatchSys / 64; ++i) a.part_mask[i] = mask[i];
  a.spin = spin;
  K1Geom geo = P->geo;
  cudaError_t e = cudaMemsetAsync(P->dbar, 0, 64, st);  // barrier and item counter
  if (e != cudaSuccess) return e;
  void* args[] = {&a, &geo};
  return cudaLaunchCooperativeKernel(cg2b_fn(geo.G4, geo.npt), dim3(geo.grid), dim3(geo.nthr * geo.G4 + 32), args,
                                     geo.smem, st);
}

cudaError_t cg2b_autotune(CG2BPlan* P, cudaStream_t st, int passes, int* chosen, float* best_us, int* tried) {
  std::vector<K1Geom> cand;
  cg2b_candidates(P, &cand);
  *chosen = -1;
  *tried = 0;
  *best_us = 0.f;
  if (cand.empty()) return cudaErrorInvalidConfiguration;
  const int nsys = (int)P->desc.size();
  unsigned long long mask[kMaxBatchSys / 64] = {0, 0, 0, 0};
  for (int s = 0; s < nsys; ++s) mask[s >> 6] |= 1ull << (s & 63);
  // every orbital active: N = Np in the system table while timing
  std::vector<int> nsave(nsys);
  for (int s = 0; s < nsys; ++s) {
    nsave[s] = P->desc[s].N;
    P->desc[s].N = P->desc[s].Np;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double tol0 = 0.0;
  for (int s = 0; s < nsys && e == cudaSuccess; ++s) {
    CGDevState* S = P->desc[s].st;
    e = cudaMemcpyAsync(&S->tol, &tol0, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&S->maxit, &passes, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->skip, 0, sizeof(int) * kMaxN, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float best = 0.f;
  for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
    if (cg2b_prepare_geo(P, cand[i]) != cudaSuccess || !P->ok) {
      (void)cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    bool ok = true;
    for (int s = 0; s < nsys && ok; ++s) ok = cudaMemsetAsync(&P->desc[s].st->status, 0, sizeof(int), st) == cudaSuccess;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      for (int s = 0; s < nsys && ok; ++s) {
        const CG2BSysDesc& d = P->desc[s];
        const long long n = (long long)d.g.nI * d.Np;
        ok = cudaMemsetAsync(d.r[0], 0, sizeof(float) * d.g.G * d.Np, st) == cudaSuccess;
        if (ok) {
          k_fill_interior_gm_b<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d.g, d.Np, d.r[0]);
          ok = cudaGetLastError() == cudaSuccess;
        }
      }
      ok = ok && cudaEventRecord(e0, st) == cudaSuccess && cg2b_launch(P, mask, kSpinLimit, st) == cudaSuccess &&
           cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    for (int s = 0; s < nsys && ok; ++s) {
      int status = 0;
      ok = cudaMemcpy(&status, &P->desc[s].st->status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
           (status & (kStatTimeout | kStatNonFinite | kStatNotSPD)) == 0;
    }
    if (!ok) {
      (void)cudaGetLastError();
      continue;
    }
    ++*tried;
    if (std::getenv("PARO_PRINT_PLAN"))
      std::fprintf(stderr, "paro batched CG candidate: tile %dx%d, %d nodes a thread, block %d, %d slots, z-chunk %d, "
                   "%d items, %.2f us a pass\n", cand[i].TX, cand[i].TY, cand[i].npt, cand[i].G4 * 4, cand[i].slots,
                   P->args.zlen, P->args.nitems, 1e3f * ms / (passes + 1));
    if (*chosen < 0 || ms < best) {
      best = ms;
      *chosen = (int)i;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int s = 0; s < nsys; ++s) {
    P->desc[s].N = nsave[s];
    const int zero = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&P->desc[s].st->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return e;
  if (*chosen < 0) return cg2b_prepare_geo(P, cand[0]);
  *best_us = 1e3f * best / (passes + 1);
  return cg2b_prepare_geo(P, cand[*chosen]);
}

}  // namespace paro
