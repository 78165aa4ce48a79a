// Single-pass Jacobi PCG for the float32 correction solves of Step 3 (the N
// independent shifted source problems A x_i = b_i of eq. 3.2, each with its own
// convergence mask), one cooperative launch per solve, one pass over the mesh
// per CG iteration and one cross-CTA reduction per pass.
//
// Textbook preconditioned CG (z = D^-1 r) with the iteration's two reductions
// merged into one: with q_k = A p_k,
//   alpha_k = rho_k / (p_k, q_k),                       rho_k = (r_k, z_k)
//   rho_{k+1} = (r_k - alpha q_k, D^-1 (r_k - alpha q_k))
//            = rho_k - 2 alpha_k (q_k, z_k) + alpha_k^2 (q_k, D^-1 q_k),
//   beta_k = rho_{k+1} / rho_k,
// so pass k, given alpha_{k-1} and beta_{k-1} from the previous reduction and
// r_{k-1}, q_{k-1}, p_{k-1} staged with a one-node halo, forms
//   r_k = r_{k-1} - alpha_{k-1} q_{k-1},  z_k = D^-1 r_k,  p_k = z_k + beta_{k-1} p_{k-1}
// at the 3 x 3 neighbours of each node (every thread for its own stencil: the
// staged data stay read-only, so no CTA barrier is needed within a plane), then
// q_k = A p_k (27-point stencil), and at its own nodes x_k = x_{k-1} +
// alpha_{k-1} p_{k-1}, and the five sums (r_k, z_k), (r_k, r_k), (p_k, q_k),
// (q_k, z_k), (q_k, D^-1 q_k).  Every pass computes rho_k from the new residual
// itself, so the expansion above only supplies beta_k and its rounding never
// accumulates.  Per unit (node x orbital) and pass the kernel reads r, q, p (with
// halo) and x, and writes r, q, p, x: 32 bytes, the method's floor.  The first
// pass (x0 = 0, r_{-1} = b, q_{-1} = p_{-1} = 0) reads only b.
//
// Vectors are group-major (cg.cuh): a converged group of four orbitals is
// neither loaded nor stored, and the threads that would handle it are whole
// idle warps (thread = node slot + nthr x active-group slot).
//
// Cross-CTA reduction: every CTA writes its partials and meets the others at a
// bounded grid barrier; the owner CTA of orbital o (o mod grid) then sums that
// orbital's partials over all CTAs in a fixed order, takes the scalar step
// (alpha, beta, convergence) and publishes it; a second barrier, and every CTA
// reads the published steps.  Each partial is read once (not by every CTA: 152
// CTAs reading the same 120 KB of partials took ~9 us a pass at 64^3 x 20), and
// the results are identical everywhere and run to run.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "cg.cuh"
#include "cgutil.cuh"
#include "tma.cuh"
#include "cg2util.cuh"

namespace paro {

namespace {

__host__ __device__ inline size_t small_state_bytes(int Np, int nob, int G4) {
  return ((size_t)2 * Np + Np / 4 + nob + (size_t)nob * G4) * 4 + 8;
}

// Fixed-order column sums of a [rows][cols] block of doubles by the nc consumer
// threads (block_colsum with the consumer barrier); sums in tmp[0 .. cols).
__device__ void consumer_colsum(const double* in, int rows, int cols, double* tmp, int nc) {
  const int t0 = threadIdx.x;
  int S = nc / cols;
  if (S < 1) S = 1;
  if (S > rows) S = rows;
  for (int t = t0; t < S * cols; t += nc) {
    const int c = t % cols, sl = t / cols;
    double a0 = 0, a1 = 0;
    int r = sl;
    for (; r + S < rows; r += 2 * S) {
      a0 += in[r * cols + c];
      a1 += in[(r + S) * cols + c];
    }
    if (r < rows) a0 += in[r * cols + c];
    tmp[t] = a0 + a1;
  }
  consumer_sync(nc);
  double v = 0.0;
  if (t0 < cols)
    for (int sl = 0; sl < S; ++sl) v += tmp[sl * cols + t0];
  consumer_sync(nc);
  if (t0 < cols) tmp[t0] = v;
  consumer_sync(nc);
}

template <int G4, int NPT>
__global__ void __launch_bounds__(cg2_max_threads(NPT), 1) k_cg2(CG2Args a, K1Geom geo, const __grid_constant__ CUtensorMap mr0,
                                                     const __grid_constant__ CUtensorMap mq0,
                                                     const __grid_constant__ CUtensorMap mp0,
                                                     const __grid_constant__ CUtensorMap mr1,
                                                     const __grid_constant__ CUtensorMap mq1,
                                                     const __grid_constant__ CUtensorMap mp1,
                                                     const __grid_constant__ CUtensorMap md,
                                                     const __grid_constant__ CUtensorMap mw) {
  constexpr int bw = 4 * G4;
  extern __shared__ __align__(128) unsigned char smem[];
  const int TX = geo.TX, TY = geo.TY;
  const int HX = TX + 2, HY = TY + 2;
  const int nthr = geo.nthr;  // TX * TY / NPT: NPT tile nodes per consumer thread
  const int NC = nthr * G4;   // consumer threads
  const int S = geo.slots;
  const int tid = threadIdx.x;
  const bool producer = tid >= NC;
  const int j = tid % nthr;   // node slot
  const int k = tid / nthr;   // active-group slot of the current orbital block (consumers)
  const int Np = a.Np;
  const long long G = a.g.G;
  const int vecf = HY * HX * 4;  // floats of one group's staged box
  const int vstr = box_stride_floats(HX, HY);  // its slot stride: TMA writes to 128-byte aligned addresses
  const unsigned spin = a.spin;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxSlots2;
  unsigned char* base = smem + 128;
  auto slotR = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes); };
  auto slotQ = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_p); };
  auto slotP = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_s); };
  auto slotD = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_d); };
  auto slotW = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * geo.slot_bytes + geo.off_w); };
  double* sacc = reinterpret_cast<double*>(base + (size_t)S * geo.slot_bytes);  // [5 Np]
  double* st_rho = sacc + kDots * Np;  // rho_k of the last reduction
  double* st_bb = st_rho + Np;         // ||b||^2
  double* st_al = st_bb + Np;          // alpha of the last reduction
  double* st_be = st_al + Np;          // beta of the last reduction
  int* st_act = reinterpret_cast<int*>(st_be + Np);
  int* st_it = st_act + Np;
  float* sbeta = reinterpret_cast<float*>(st_it + Np);  // [Np] beta and alpha of the pass, float32
  float* salpha = sbeta + Np;
  int* sgact = reinterpret_cast<int*>(salpha + Np);      // [Np/4] group still iterating
  int* snact = sgact + Np / 4;                            // [nob] active groups per orbital block
  int* slist = snact + geo.nob;                           // [nob G4] the blocks' active groups in order
  double* sred = reinterpret_cast<double*>(smem_align8(slist + geo.nob * G4));  // sums / reduction scratch
  __shared__ int s_nact, s_ok, s_lstep;

  const int nzo = a.g.nz - 1;
  const long long fbeg = geo.split[blockIdx.x];
  const long long fend = geo.split[blockIdx.x + 1];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC / 32);
    }
    fence_mbar_init();
  }
  if (tid == NC) {
    prefetch_tmap(&mr0);
    prefetch_tmap(&mq0);
    prefetch_tmap(&mp0);
    prefetch_tmap(&mr1);
    prefetch_tmap(&mq1);
    prefetch_tmap(&mp1);
    prefetch_tmap(&md);
    prefetch_tmap(&mw);
  }
  const int maxit = a.st->maxit;
  const double tol = a.st->tol;
  for (int o = tid; o < Np; o += blockDim.x) {
    st_rho[o] = 0.0;
    st_bb[o] = 0.0;
    st_al[o] = 0.0;
    st_be[o] = 0.0;
    st_act[o] = (o < a.N && a.st->skip[o] == 0 && maxit > 0) ? 1 : 0;
    st_it[o] = 0;
  }
  __syncthreads();

  auto seg_at = [&](long long f, int& o0, int& x0, int& y0, int& z0, int& z1) {
    const long long col = f / nzo;
    const int zl = (int)(f - col * nzo);
    const long long rem = fend - f;
    const int zh = (rem < (long long)(nzo - zl)) ? zl + (int)rem : nzo;
    const int tx = (int)(col % geo.ncx);
    const long long r = col / geo.ncx;
    const int ty = (int)(r % geo.ncy);
    const int ob = (int)(r / geo.ncy);
    o0 = ob * bw;
    x0 = 1 + tx * TX;
    y0 = 1 + ty * TY;
    z0 = 1 + zl;
    z1 = 1 + zh;
  };

  const uint32_t vbytes = (uint32_t)vecf * 4u;
  const uint32_t dwbytes = (uint32_t)(geo.DX * HY + kW2 * TX * TY) * 4u;
  bool first = true;  // pass 0: only b is read
  int rd = 0;         // buffer set read by the current pass
  int lstep = 0;      // producer: planes staged so far (all passes)
  int cstep = 0;      // consumers: planes consumed so far

  // producer (one lane): stage every input plane of this CTA's pass, waiting for
  // a slot to be released before reusing it; false on a timed-out wait
  auto produce = [&]() -> bool {
    const CUtensorMap* R = rd ? &mr1 : &mr0;
    const CUtensorMap* Q = rd ? &mq1 : &mq0;
    const CUtensorMap* P = rd ? &mp1 : &mp0;
    for (long long f = fbeg; f < fend;) {
      int o0, x0, y0, z0, z1;
      seg_at(f, o0, x0, y0, z0, z1);
      f += z1 - z0;
      const int ob = o0 / bw;
      const int na = snact[ob];
      if (na == 0) continue;
      for (int zin = z0 - 1; zin <= z1; ++zin) {
        const int slot = lstep % S;
        if (lstep >= S && !mbar_wait_n(&empty[slot], ((lstep / S) - 1) & 1, spin)) return false;
        mbar_arrive_expect_tx(&full[slot], (uint32_t)na * (first ? 1u : 3u) * vbytes + dwbytes);
        for (int kk = 0; kk < na; ++kk) {
          const int gam = slist[ob * G4 + kk];
          tma_load_4d(slotR(slot) + kk * vstr, R, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
          if (!first) {
            tma_load_4d(slotQ(slot) + kk * vstr, Q, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
            tma_load_4d(slotP(slot) + kk * vstr, P, 4 * (x0 - 1), y0 - 1, zin, gam, &full[slot]);
          }
        }
        tma_load_3d(slotD(slot), &md, x0 - 1, y0 - 1, zin, &full[slot]);
        tma_load_4d(slotW(slot), &mw, 0, x0 - 1, y0 - 1, zin, &full[slot]);
        ++lstep;
      }
    }
    return true;
  };

  // own nodes (tx, ty0 + i), i < NPT, of the tile
  const int tx = j % TX, ty0 = (j / TX) * NPT;
  const long long plane = (long long)a.g.Px * a.g.Py;
  const int lane = tid & 31;

  bool timed_out = false;
  int status = 0;

  // adds the consumers' per-orbital sums of the block's active groups into sacc: a
  // float32 butterfly over the 32 node slots of each warp (a warp holds one group
  // slot: nthr is a multiple of 32), then the warps of a group slot in order, in
  // float64 (two consumer barriers, the order fixed)
  auto flush = [&](int ob, int na, float (&dt)[kDots][4]) {
    const int wpg = nthr >> 5;
#pragma unroll
    for (int d = 0; d < kDots; ++d)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v = dt[d][c];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        dt[d][c] = v;
      }
    if (lane == 0 && k < na) {
#pragma unroll
      for (int d = 0; d < kDots; ++d)
#pragma unroll
        for (int c = 0; c < 4; ++c) sred[(tid >> 5) * (kDots * 4) + d * 4 + c] = (double)dt[d][c];
    }
    consumer_sync(NC);
    for (int t = tid; t < kDots * 4 * na; t += NC) {
      const int kk = t / (kDots * 4), e = t - kk * (kDots * 4);
      double v = 0.0;
      for (int q = 0; q < wpg; ++q) v += sred[(kk * wpg + q) * (kDots * 4) + e];
      sacc[(e >> 2) * Np + 4 * slist[ob * G4 + kk] + (e & 3)] += v;
    }
    consumer_sync(NC);
  };

  // consumers: one pass over this CTA's column-planes; false on a timed-out wait.
  // No CTA barrier per plane: every thread forms p_k = D^-1 (r - alpha q) + beta p
  // itself at the 3 x 3 neighbours its stencil reads (the staged slot is never
  // written), so warps only meet at the ring's mbarriers.  After a timed-out wait a
  // thread stops waiting and computing but keeps to the loop, so the consumer
  // barriers of the flush are still reached by everyone.
  auto consume = [&]() -> bool {
    float* const wx = a.x;
    float* const wr = a.r[rd ^ 1];
    float* const wq = a.q[rd ^ 1];
    float* const wp = a.p[rd ^ 1];
    bool ok = true;
    int cur_ob = -1, cur_na = 0;
    float dt[kDots][4];
#pragma unroll
    for (int d = 0; d < kDots; ++d)
#pragma unroll
      for (int c = 0; c < 4; ++c) dt[d][c] = 0.f;
    for (long long f = fbeg; f < fend;) {
      int o0, x0, y0, z0, z1;
      seg_at(f, o0, x0, y0, z0, z1);
      f += z1 - z0;
      const int ob = o0 / bw;
      const int na = snact[ob];
      if (na == 0) continue;
      if (ob != cur_ob) {
        if (cur_ob >= 0) {
          flush(cur_ob, cur_na, dt);
#pragma unroll
          for (int d = 0; d < kDots; ++d)
#pragma unroll
            for (int c = 0; c < 4; ++c) dt[d][c] = 0.f;
        }
        cur_ob = ob;
        cur_na = na;
      }
      const bool kact = k < na;
      const int gam = kact ? slist[ob * G4 + k] : 0;
      float al[4], be[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        al[c] = kact ? salpha[4 * gam + c] : 0.f;
        be[c] = kact ? sbeta[4 * gam + c] : 0.f;
      }
      const int xg = x0 + tx;
      const long long gbase = (long long)gam * G;
      bool inside[NPT];
      long long colnode[NPT];
      Vec4<float> aU[NPT], aC[NPT], aD[NPT];
      Vec4<float> pv_z[NPT], pv_p[NPT];  // own nodes' z_k and p_k of the previous input plane
      float pv_d[NPT];
      Vec4<float> xnext[NPT];             // x of the next plane, loaded one plane ahead
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        const int yg = y0 + ty0 + i;
        inside[i] = xg <= a.g.nx - 1 && yg <= a.g.ny - 1;
        colnode[i] = (long long)yg * a.g.Px + xg;
        aU[i] = aC[i] = aD[i] = pv_z[i] = pv_p[i] = xnext[i] = Vec4<float>{};
        pv_d[i] = 0.f;
      }
      for (int s = z0 - 1; s <= z1; ++s) {
        const int slot = cstep % S;
        const uint32_t par = (cstep / S) & 1;
        const bool zout = s >= z0 && s < z1;
        long long eown[NPT];
        Vec4<float> xv[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          eown[i] = (gbase + (long long)s * plane + colnode[i]) * 4;
          xv[i] = xnext[i];
          if (ok && !first && kact && inside[i] && s + 1 >= z0 && s + 1 < z1) xnext[i] = ldcg4(wx + eown[i] + plane * 4);
        }
        if (ok) ok = mbar_wait_n(&full[slot], par, spin);
        Vec4<float> cz[NPT], cp[NPT];
        float cd[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          cz[i] = cp[i] = Vec4<float>{};
          cd[i] = 0.f;
        }
        if (kact && ok) {
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
          // the staged rows ty0 .. ty0 + NPT + 1 (halo-relative), columns tx - 1 .. tx + 1:
          // every node's r_k, z_k, p_k once, then its weight in each own node's stencil
#pragma unroll
          for (int cy = 0; cy < NPT + 2; ++cy) {
#pragma unroll
            for (int cxi = 0; cxi < 3; ++cxi) {
              const int hnode = (ty0 + cy) * HX + (tx + cxi);
              const int e = hnode * 4;
              const float d = D[(ty0 + cy) * geo.DX + tx + cxi];
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
                if (cyr == 1 && cxi == 1) {  // own node i: r_k, p_k, x_k and their sums
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
                    sts4(wr + eown[i], rn);
                    sts4(wp + eown[i], pn);
                    sts4(wx + eown[i], xn);
                  }
                }
              }
            }
          }
        }
        // this warp is done with the slot
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(&empty[slot]);
        if (kact) {
#pragma unroll
          for (int i = 0; i < NPT; ++i) {
            // output plane s-1 is complete: q_k there, and its sums
            const bool prev_out = ok && inside[i] && s - 1 >= z0 && s - 1 < z1;
            if (prev_out) {
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                dt[2][c] = fmaf(pv_p[i].v[c], aD[i].v[c], dt[2][c]);
                dt[3][c] = fmaf(aD[i].v[c], pv_z[i].v[c], dt[3][c]);
                dt[4][c] = fmaf(aD[i].v[c], pv_d[i] * aD[i].v[c], dt[4][c]);
              }
              sts4(wq + eown[i] - plane * 4, aD[i]);
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
      }
    }
    if (cur_ob >= 0) flush(cur_ob, cur_na, dt);
    return ok;
  };

  // masks of the next pass: group and block activity, the active-group lists
  auto load_masks = [&]() {
    for (int o = tid; o < Np; o += blockDim.x) {
      sbeta[o] = (float)st_be[o];
      salpha[o] = (float)st_al[o];
    }
    for (int q = tid; q < Np / 4; q += blockDim.x)
      sgact[q] = st_act[4 * q] | st_act[4 * q + 1] | st_act[4 * q + 2] | st_act[4 * q + 3];
    __syncthreads();
    for (int ob = tid; ob < geo.nob; ob += blockDim.x) {
      int n = 0;
      for (int q = ob * G4; q < ob * G4 + G4 && q < Np / 4; ++q)
        if (sgact[q]) slist[ob * G4 + n++] = q;
      snact[ob] = n;
    }
    __syncthreads();
  };

  // bounded grid barrier: arrival `target` of the launch's counter
  auto grid_sync = [&](unsigned target) -> bool {
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      atomicAdd(&a.st->bar_count, 1u);
      int okb = 0;
      for (unsigned i = 0; i < spin; ++i) {
        if (ld_acquire_u32(&a.st->bar_count) >= target) {
          okb = 1;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
      s_ok = okb;
    }
    __syncthreads();
    return s_ok != 0;
  };
  for (int npass = 0;; ++npass) {
    if (tid == 0) s_nact = 0;
    __syncthreads();
    for (int o = tid; o < Np; o += blockDim.x)
      if (st_act[o]) atomicAdd(&s_nact, 1);
    __syncthreads();
    const int nact_orb = s_nact;
    if (nact_orb == 0) break;
    load_masks();
    if (blockIdx.x == 0 && tid == 0) {
      unsigned long long ng = 0, nb = 0;
      for (int ob = 0; ob < geo.nob; ++ob) {
        ng += (unsigned long long)snact[ob];
        if (snact[ob]) ++nb;
      }
      a.st->work += 4ull * ng * (unsigned long long)a.g.nI;
      a.st->work_nodes += nb * (unsigned long long)a.g.nI;
      a.st->work_act += (unsigned long long)nact_orb * (unsigned long long)a.g.nI;
    }
    for (int o = tid; o < kDots * Np; o += blockDim.x) sacc[o] = 0.0;
    __syncthreads();
    bool ok = true;
    if (producer) {
      if (tid == NC) {
        fence_proxy_async_global2();  // the previous pass's generic stores before this pass's TMA reads
        ok = produce();
      }
      __syncwarp();  // the producer warp reconverges before the CTA barrier
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
    // partials of this CTA as [o][d][CTA], then the first bounded grid barrier (the
    // owners read them before the second one, which every CTA passes before it
    // writes the next pass's)
    const unsigned nG = gridDim.x;
    double* part = a.part + (long long)(npass & 1) * kDots * nG * Np;
    for (int t = tid; t < kDots * Np; t += blockDim.x) {
      const int d = t / Np, o = t - d * Np;
      part[((long long)o * kDots + d) * nG + blockIdx.x] = sacc[t];
    }
    fence_proxy_async_global2();  // this pass's generic stores before the next pass's TMA reads
    if (!grid_sync((2u * npass + 1u) * nG)) {
      timed_out = true;
      break;
    }
    // the owner of each still-iterating orbital: its five sums over the CTAs (one
    // warp a sum, lanes over CTAs, then a butterfly), the scalar step, published
    double* pub = a.pub + (long long)(npass & 1) * 4 * Np;
    const int nwarp = blockDim.x >> 5;
    for (int o = blockIdx.x; o < Np; o += nG) {
      if (!st_act[o]) continue;  // the same for the whole CTA
      for (int d = tid >> 5; d < kDots; d += nwarp) {
        const double* src = part + ((long long)o * kDots + d) * nG;
        double v = 0.0;
#pragma unroll 4
        for (unsigned c = lane; c < nG; c += 32) v += __ldcg(src + c);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) sred[d] = v;
      }
      __syncthreads();
      if (tid == 0) {
        const double rho = sred[0], rr = sred[1], pq = sred[2], qz = sred[3], qdq = sred[4];
        bool act = true;
        double alpha = 0.0, beta = 0.0;
        if (npass == 0) {
          st_bb[o] = rr;  // r_0 = b
        } else {
          st_it[o] += 1;  // x was updated in this pass
          a.st->rr[o] = rr;
        }
        if (!(isfinite(rho) && isfinite(rr) && isfinite(pq) && isfinite(qz) && isfinite(qdq))) {
          status |= kStatNonFinite;
          act = false;
        } else if (npass > 0 && rr <= tol * tol * st_bb[o]) {
          act = false;
        } else if (npass > 0 && st_it[o] >= maxit) {
          if (!a.inner) status |= kStatNotConverged;
          act = false;
        }
        if (act) {
          if (!(rho > 0.0) || !(pq > 0.0)) {
            status |= kStatNotSPD;
            act = false;
          } else {
            alpha = rho / pq;
            const double rho1 = rho - 2.0 * alpha * qz + alpha * alpha * qdq;
            beta = rho1 > 0.0 ? rho1 / rho : 0.0;
          }
        }
        st_rho[o] = rho;
        pub[4 * o] = act ? alpha : 0.0;
        pub[4 * o + 1] = act ? beta : 0.0;
        pub[4 * o + 2] = act ? 1.0 : 0.0;
      }
      __syncthreads();
    }
    if (!grid_sync((2u * npass + 2u) * nG)) {
      timed_out = true;
      break;
    }
    for (int o = tid; o < Np; o += blockDim.x) {
      if (!st_act[o]) {
        st_al[o] = 0.0;
        st_be[o] = 0.0;
        continue;
      }
      st_al[o] = __ldcg(pub + 4 * o);
      st_be[o] = __ldcg(pub + 4 * o + 1);
      st_act[o] = __ldcg(pub + 4 * o + 2) != 0.0 ? 1 : 0;
    }
    __syncthreads();
  }
  if (timed_out) {
    // every consumer stopped at the same plane (cstep); the copies staged beyond
    // it land before the CTA exits (bounded, at the full limit)
    if (tid == 0) {
      atomicOr(&a.st->status, kStatTimeout);
      for (int q = cstep; q < s_lstep; ++q) mbar_wait_n(&full[q % S], (q / S) & 1, kSpinLimit);
    }
  }
  if (status) atomicOr(&a.st->status, status);
  __syncthreads();
  // the owners: their orbitals' iteration counts and ||b||^2; CTA 0: the flags
  if (tid == 0) {
    long long isum = 0;
    int imax = 0;
    for (int o = blockIdx.x; o < Np; o += gridDim.x) {
      a.st->iters[o] = st_it[o];
      a.st->bb[o] = st_bb[o];
      isum += st_it[o];
      imax = st_it[o] > imax ? st_it[o] : imax;
    }
    if (isum) atomicAdd(reinterpret_cast<unsigned long long*>(&a.st->it_sum), (unsigned long long)isum);
    if (imax) atomicMax(&a.st->it_max, imax);
  }
  if (blockIdx.x == 0) {
    if (tid == 0) s_nact = 0;
    __syncthreads();
    for (int o = tid; o < Np; o += blockDim.x) {
      a.st->active[o] = st_act[o];
      if (st_act[o]) atomicAdd(&s_nact, 1);
    }
    __syncthreads();
    if (tid == 0) a.st->n_active = s_nact;
  }
}

template <int NPT>
void* cg2_fn_npt(int G4) {
  switch (G4) {
    case 1: return (void*)k_cg2<1, NPT>;
    case 2: return (void*)k_cg2<2, NPT>;
    case 3: return (void*)k_cg2<3, NPT>;
    case 4: return (void*)k_cg2<4, NPT>;
    case 5: return (void*)k_cg2<5, NPT>;
    case 6: return (void*)k_cg2<6, NPT>;
    case 7: return (void*)k_cg2<7, NPT>;
    case 8: return (void*)k_cg2<8, NPT>;
  }
  return nullptr;
}

void* cg2_fn(int G4, int npt) { return npt == 2 ? cg2_fn_npt<2>(G4) : npt == 1 ? cg2_fn_npt<1>(G4) : nullptr; }

// b = 1 at the interior nodes of every group (boundary rows stay zero), group-major
__global__ void k_fill_interior_gm(Grid g, int Np, float* b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * Np) return;
  const int o = (int)(t % Np);
  const long long gp = interior_to_padded(g, (int)(t / Np));
  b[((long long)(o / 4) * g.G + gp) * 4 + o % 4] = 1.0f;
}

}  // namespace

// Shared-memory footprint: a ring of slots of r, q, p boxes for up to G4 groups
// (each [TY+2][TX+2][4], 128-byte aligned), D^-1 [TY+2][DX] and the packed
// weights [TY][TX][28]; then the sums [5 Np], per-orbital state (4 Np doubles,
// 2 Np ints), the flush's per-warp sums and an owner's five totals.  The ring takes as many
// slots (3 to 6) as fit in `limit` bytes; false if not even 3 do.
static bool cg2_layout(int Np, int bw, int TX, int TY, int npt, size_t limit, K1Geom* G) {
  const size_t sz = sizeof(float);
  const int G4 = bw / 4;
  G->TX = TX;
  G->TY = TY;
  G->npt = npt;
  G->nthr = TX * TY / npt;
  const int HX = TX + 2, HY = TY + 2;
  G->DX = TX + 4;
  const size_t vec = (size_t)G4 * box_stride_floats(HX, HY) * sz;
  const size_t dv = (size_t)G->DX * HY * sz;
  const size_t wv = (size_t)kW2 * TX * TY * sz;
  auto al = [](size_t v) { return (v + 127) / 128 * 128; };
  G->off_p = (int)al(vec);                 // q boxes
  G->off_s = (int)(G->off_p + al(vec));    // p boxes
  G->off_d = (int)(G->off_s + al(vec));
  G->off_w = (int)(G->off_d + al(dv));
  G->slot_bytes = (int)(G->off_w + al(wv));
  G->tx_bytes = (uint32_t)(3 * (size_t)G4 * HX * HY * 16 + dv + wv);  // all groups active
  const size_t nt = (size_t)G->nthr * G4 + 32;
  const size_t wsum = (nt - 32) / 32 * kDots * 4 + 8;  // flush: per-warp sums; an owner's five totals
  const int nob = (Np + bw - 1) / bw;
  const size_t red = ((size_t)kDots * Np + 4 * (size_t)Np + Np + wsum) * sizeof(double) +
                     small_state_bytes(Np, nob, G4);
  if (128 + red + 3 * (size_t)G->slot_bytes > limit) return false;
  int slots = (int)((limit - 128 - red) / G->slot_bytes);
  if (slots > kMaxSlots2) slots = kMaxSlots2;
  G->slots = slots;
  G->smem = 128 + (size_t)slots * G->slot_bytes + red;
  return true;
}

static void cg2_finish(const Grid& g, int Np, int nsm, int bw, K1Geom* G) {
  G->G4 = bw / 4;
  G->ncx = (g.nx - 1 + G->TX - 1) / G->TX;
  G->ncy = (g.ny - 1 + G->TY - 1) / G->TY;
  G->nob = (Np + bw - 1) / bw;
  long long want = nsm;  // one CTA per SM (all co-resident)
  if (want > kMaxGrid1) want = kMaxGrid1;
  const long long F = (long long)G->nob * G->ncx * G->ncy * (g.nz - 1);
  long long grid = F / 4;
  if (grid < 1) grid = 1;
  if (grid > want) grid = want;
  G->grid = (int)grid;
  balanced_split(F, g.nz - 1, G->grid, G->split);
}

void cg2_candidates(const Grid& g, int Np, int nsm, std::vector<K1Geom>* out) {
  out->clear();
  const size_t stat = 64;  // the kernel's static shared memory (a few ints)
  const size_t limit = 227 * 1024 - stat - 1024;
  // tiles of 64 or 96 nodes (two or three warps per group slot): the larger ones
  // stage fewer halo nodes per node (1.5x at 16 x 6 against 1.69x at 16 x 4) and
  // run more warps per SM (32-node tiles at two CTAs a SM measured slower)
  // (TX, TY, nodes a thread): the two-node slots take taller tiles (128 nodes: 1.41
  // staged nodes a node against 1.5-1.69 for the 64- and 96-node tiles)
  const int shapes[8][3] = {{16, 4, 1}, {8, 8, 1}, {16, 6, 1}, {24, 4, 1}, {8, 12, 1},
                            {16, 8, 2}, {32, 4, 2}, {8, 16, 2}};
  int widths = 0;
  for (int nob = (Np + 31) / 32; nob <= Np / 4 && widths < 3; ++nob) {
    int bw = (Np + nob - 1) / nob;
    bw = (bw + 3) / 4 * 4;
    if ((Np + bw - 1) / bw != nob) continue;
    bool any = false;
    for (int si = 0; si < 8; ++si) {
      const int TX = shapes[si][0], TY = shapes[si][1], npt = shapes[si][2];
      if (TX * TY / npt * (bw / 4) + 32 > cg2_max_threads(npt)) continue;  // consumers + the producer warp
      K1Geom G{};
      if (!cg2_layout(Np, bw, TX, TY, npt, limit, &G)) continue;
      cg2_finish(g, Np, nsm, bw, &G);
      out->push_back(G);
      any = true;
    }
    if (any) ++widths;
  }
}

cudaError_t cg2_prepare_geo(CG2Plan* P, const K1Geom& geo) {
  cudaError_t e;
  P->ok = false;
  P->geo = geo;
  const K1Geom& G = P->geo;
  const CG2Args& a = P->args;
  const uint64_t sz = sizeof(float);
  const CUtensorMapDataType ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  {
    // group-major vector as (4 Px, Py, Pz, Np/4): a box row is 4 (TX+2) contiguous floats
    uint64_t dims[4] = {(uint64_t)4 * a.g.Px, (uint64_t)a.g.Py, (uint64_t)a.g.Pz, (uint64_t)(a.Np / 4)};
    uint64_t str[3] = {(uint64_t)4 * a.g.Px * sz, (uint64_t)4 * a.g.Px * a.g.Py * sz, (uint64_t)4 * a.g.G * sz};
    uint32_t box[4] = {(uint32_t)(4 * (G.TX + 2)), (uint32_t)(G.TY + 2), 1, 1};
    for (int s = 0; s < 2; ++s) {
      if ((e = encode_tiled(&P->mr[s], ty, 4, a.r[s], dims, str, box)) != cudaSuccess) return e;
      if ((e = encode_tiled(&P->mq[s], ty, 4, a.q[s], dims, str, box)) != cudaSuccess) return e;
      if ((e = encode_tiled(&P->mp[s], ty, 4, a.p[s], dims, str, box)) != cudaSuccess) return e;
    }
  }
  {
    uint64_t dims[3] = {(uint64_t)P->dpitch, (uint64_t)a.g.Py, (uint64_t)a.g.Pz};
    uint64_t str[2] = {(uint64_t)P->dpitch * sz, (uint64_t)P->dpitch * a.g.Py * sz};
    uint32_t box[3] = {(uint32_t)G.DX, (uint32_t)(G.TY + 2), 1};
    if ((e = encode_tiled(&P->md, ty, 3, (void*)P->dinv_tma, dims, str, box)) != cudaSuccess) return e;
  }
  {
    const uint64_t nxi = (uint64_t)(a.g.nx - 1), nyi = (uint64_t)(a.g.ny - 1);
    uint64_t dims[4] = {(uint64_t)kW2, nxi, nyi, (uint64_t)a.g.Pz};
    uint64_t str[3] = {(uint64_t)kW2 * sz, (uint64_t)kW2 * nxi * sz, (uint64_t)kW2 * nxi * nyi * sz};
    uint32_t box[4] = {(uint32_t)kW2, (uint32_t)G.TX, (uint32_t)G.TY, 1};
    if ((e = encode_tiled(&P->mw, ty, 4, (void*)P->wcoef, dims, str, box)) != cudaSuccess) return e;
  }
  void* f = cg2_fn(G.G4, G.npt);
  if (!f) return cudaErrorInvalidValue;
  if ((e = allow_max_dyn_smem(f)) != cudaSuccess) return e;
  int nb = 0, dev = 0, coop = 0;
  P->ok = cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, G.nthr * G.G4 + 32, G.smem) == cudaSuccess &&
          (long long)nb * P->nsm >= G.grid;
  (void)cudaGetLastError();
  return cudaSuccess;
}

cudaError_t cg2_launch(CG2Plan* P, cudaStream_t st) {
  CG2Args a = P->args;
  K1Geom geo = P->geo;
  cudaError_t e = cudaMemsetAsync(&a.st->bar_count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  void* args[] = {&a, &geo, &P->mr[0], &P->mq[0], &P->mp[0], &P->mr[1], &P->mq[1], &P->mp[1], &P->md, &P->mw};
  return cudaLaunchCooperativeKernel(cg2_fn(geo.G4, geo.npt), dim3(geo.grid), dim3(geo.nthr * geo.G4 + 32), args, geo.smem,
                                     st);
}

cudaError_t cg2_autotune(CG2Plan* P, cudaStream_t st, int passes, int* chosen, float* best_us, int* tried) {
  std::vector<K1Geom> cand;
  cg2_candidates(P->args.g, P->args.Np, P->nsm, &cand);
  *chosen = -1;
  *tried = 0;
  *best_us = 0.f;
  if (cand.empty()) return cudaErrorInvalidConfiguration;
  CG2Args& a = P->args;
  const int Nsave = a.N, inner = a.inner;
  a.N = a.Np;
  a.inner = 1;
  const double tol0 = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&a.st->tol, &tol0, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&a.st->maxit, &passes, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.st->skip, 0, sizeof(int) * kMaxN, st);
  const long long n = (long long)a.g.nI * a.Np;
  float best = 0.f;
  for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
    if (cg2_prepare_geo(P, cand[i]) != cudaSuccess || !P->ok) {
      (void)cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    bool ok = cudaMemsetAsync(&a.st->status, 0, sizeof(int), st) == cudaSuccess;
    for (int rep = 0; rep < 4 && ok; ++rep) {  // a warm-up run, then the best of three timed runs
      // b = 1 (the first pass reads it from set 0, later passes overwrite it)
      ok = cudaMemsetAsync(a.r[0], 0, sizeof(float) * a.g.G * a.Np, st) == cudaSuccess;
      if (ok) {
        k_fill_interior_gm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.g, a.Np, a.r[0]);
        ok = cudaGetLastError() == cudaSuccess;
      }
      float t = 0.f;
      ok = ok && cudaEventRecord(e0, st) == cudaSuccess && cg2_launch(P, st) == cudaSuccess &&
           cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
      if (rep == 1 || (rep > 1 && t < ms)) ms = t;
    }
    int status = 0;
    ok = ok && cudaMemcpy(&status, &a.st->status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
         (status & (kStatTimeout | kStatNonFinite | kStatNotSPD)) == 0;
    if (!ok) {
      (void)cudaGetLastError();
      continue;
    }
    ++*tried;
    if (std::getenv("PARO_PRINT_PLAN"))
      std::fprintf(stderr, "paro single-pass CG candidate: tile %dx%d, %d nodes a thread, block %d, %d slots, "
                   "%.2f us a pass\n", cand[i].TX, cand[i].TY, cand[i].npt, cand[i].G4 * 4, cand[i].slots,
                   1e3f * ms / (passes + 1));
    if (*chosen < 0 || ms < best) {
      best = ms;
      *chosen = (int)i;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  a.N = Nsave;
  a.inner = inner;
  const int zero = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&a.st->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (*chosen < 0) return cg2_prepare_geo(P, cand[0]);
  *best_us = 1e3f * best / (passes + 1);
  return cg2_prepare_geo(P, cand[*chosen]);
}

}  // namespace paro
