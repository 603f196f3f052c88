// aa_batch.cu -- many independent Anderson solves in one persistent launch.
//
// Workload: nonlinear-Jacobi fixed points of the 2D Bratu problem
// (Sec. 5.2 of the paper) on s x s grids of different sizes,
//   G(u)_p = (sum of the 4 neighbours + h^2 (lambda e^{u_p} + src_p)) / 4,
// h = 1/(s+1), zero boundary, each solved by AA(m) with ICWY QR updates
// (Algorithm 4; the variant the paper recommends on GPUs).
//
// Design: a persistent grid; each CTA pops the next solve from an atomic
// queue (solves sorted largest first for load balance) and runs the whole
// Anderson loop for it with block-level reductions (fixed order, so results
// are bit-reproducible), then pops the next one.  Per iteration: pass A
// evaluates G (the stencil reads x with its halo), forms f, Delta f, Delta g,
// applies the QRDelete rotation and accumulates the first block of dot
// products; warp 0 updates R and T; the projection pass forms the new
// column; warp 0 solves for gamma; the update pass writes x_{i+1}.
// Q and dG are stored in FP32 (the precision form) and the n-space arithmetic
// on them runs in FP32 (the rotation with float multipliers; projection and
// update sums with (hi, lo) float coefficients, each part in its own chain);
// dot products are exact float products summed in compensated float pairs
// and folded into FP64 (aa_df.cuh); x, G(x), f, Delta f stay FP64, and R, T,
// gamma are FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/aa.h"
#include "aa_df.cuh"

namespace {

using aa::F2;

constexpr int BM = 16;             // largest history depth of the batched form
constexpr int BNDOT = 3 + 3 * BM;  // dot products of pass A at most (state arrays)

struct Solve {
  int64_t off;     // first row in the arena
  int32_t s;       // grid side (n = s*s)
  int32_t orig;    // index in the caller's order
  double lambda;
  double scale;    // ||G(0)||_2, the stopping scale (independent of x_0)
};

struct Result {
  int32_t iters;     // iterations taken (x_0 is iterate 0)
  int32_t status;    // 0 converged, 1 iteration cap reached, AA_ENONFINITE
  double resid;      // ||f||/||G(0)|| at exit
  int32_t fallback;  // 1 if the given x_0 was replaced by 0
  int32_t pad;
  uint64_t t0, t1;   // device global timer (ns) when the solve started and stopped
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct BArgs {
  const Solve *solves;
  Result *res;
  int count;
  int m;
  int max_iters;
  double tol;
  double breakdown_tol;
  double *X0, *X1, *GP, *FP, *DF;  // FP64 vectors (arena rows)
  float *Q, *DG;                    // m slots of N floats each
  int64_t N;                        // arena rows
  const double *src;                // optional source term (arena rows) or null
  int warm;                         // x_0 given: fall back to 0 if ||f_0|| >= ||G(0)||
  unsigned *queue;                  // next solve
};

// ---------------------------------------------------------------- state

struct SState {
  double R[BM * BM], T[BM * BM], Rn[BM * BM], Tn[BM * BM];
  double sig[BM], rhs[BM], rcol[BM], coef[BM], gam[BM], gphys[BM];
  double rot[4 * BM];
  double red[BNDOT];
  double scale, vscale, fn2, dfn2;
  int c, head, pend, done, status, restarts, it, solve, fallback;
  unsigned gmask;
};

// Block reduction of nd (hi, lo) float pairs per thread into st.red.  The
// warp stage combines the pairs on the FP32 pipe (TwoSum butterfly); the
// per-warp results are folded into FP64 by one thread per value, in warp
// order (fixed, so the sums are bit-reproducible).
template <int NT, int ND>
__device__ void block_reduce_df(const float (&S)[ND], const float (&C)[ND], int nd, float2 *wbuf,
                                SState &st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    if (d < nd) {
      float s = S[d], c = C[d];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        float hs, ts;
        aa::two_sum(s, s2, hs, ts);
        ts = __fadd_rn(ts, __fadd_rn(c, c2));
        const F2 r = aa::fast_two_sum(hs, ts);
        s = r.h;
        c = r.l;
      }
      if (lane == 0) wbuf[warp * BNDOT + d] = make_float2(s, c);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nd; d += NT) {
    double v = 0.0;
    for (int w = 0; w < NW; ++w) {
      const float2 p = wbuf[w * BNDOT + d];
      v += aa::f2d(p.x);
      v += aa::f2d(p.y);
    }
    st.red[d] = v;
  }
  __syncthreads();
}

// Software prefetch into L2 of the rows a warp will stream PF row blocks
// later: lane l < ncols takes FP32 column l (one 128-byte line per 32 rows),
// lanes 16-23 take up to four FP64 vectors (two lines each).  The batched
// passes are bound by the latency of their global loads (each thread works
// through long dependency chains between its loads), and this keeps the next
// blocks' lines on their way without spending registers.
constexpr int PF = 2;

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_rows(int lane, int64_t rb, int64_t n, const float *Q,
                                              int64_t ldq, int ncols, const double *v0,
                                              const double *v1, const double *v2,
                                              const double *v3) {
  if (rb >= n) return;
  if (lane < ncols) {
    prefetch_l2(Q + (int64_t)lane * ldq + rb);
  } else if (lane >= 16 && lane < 24) {
    const int w = (lane - 16) >> 1;
    const int64_t h = (lane & 1) ? 16 : 0;
    const double *v = w == 0 ? v0 : (w == 1 ? v1 : (w == 2 ? v2 : v3));
    if (v && rb + h < n) prefetch_l2(v + rb + h);
  }
}

// Per-thread asynchronous copies (cp.async) of the next row block's
// streamed operands into a two-stage shared-memory buffer: each thread
// copies, and later reads, only its own slots, so a per-thread wait on the
// older copy group is the only synchronisation needed.
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Staging buffer bytes: 2 stages x NT threads x (4 doubles + MB floats).
__host__ __device__ constexpr size_t stage_bytes(int nt, int mb) {
  return (size_t)2 * nt * (4 * sizeof(double) + mb * sizeof(float));
}

// The m x m work below runs on warp 0 with one lane per row or column
// (m <= BM <= 32): on GB300 a warp-wide FP64 instruction costs the same
// pipe time whether one lane or all are active, so spreading the O(m^2)
// loops over the lanes cuts their time by about m.

// Warp 0: Givens parameters of the next QRDelete from R alone, in the scaled
// two-multiply-add form, plus the rotated R and ICWY's rotated T (as in the
// single-solve path).
__device__ void prepare_delete_b(SState &st, int M, int lane) {
  // Rn = R without its first column; Tn = the Gram of the stored columns
  // 0..M-2 rebuilt from T = I + L (strict lower part mirrored).
  for (int i = lane; i < BM * BM; i += 32) {
    const int j = i / BM, l = i % BM;
    st.Rn[i] = (j < M && l + 1 < M) ? st.R[j * BM + l + 1] : 0.0;
    double g = (j == l && j < M) ? 1.0 : 0.0;
    if (j != l && j < M - 1 && l < M - 1) g = (j > l) ? st.T[j * BM + l] : st.T[l * BM + j];
    st.Tn[i] = g;
  }
  __syncwarp();
  double tau = st.sig[0];  // every lane carries the same value
  for (int j = 0; j + 1 < M; ++j) {
    const double av = st.Rn[j * BM + j], bv = st.Rn[(j + 1) * BM + j];
    // one reciprocal square root on the dependency chain; hypot and
    // divisions only outside the normal range of a^2 + b^2
    const double t2 = fma(av, av, bv * bv);
    double c = 1.0, s = 0.0;
    if (t2 > 1e-290 && t2 < 1e290) {
      const double ri = rsqrt(t2);
      c = av * ri;
      s = bv * ri;
    } else if (av != 0.0 || bv != 0.0) {
      const double rho = hypot(av, bv);
      c = av / rho;
      s = bv / rho;
    }
    __syncwarp();
    {
      const int l = j + lane;  // rows j, j+1 over columns j..M-2
      if (l + 1 < M) {
        const double hj = st.Rn[j * BM + l], hj1 = st.Rn[(j + 1) * BM + l];
        st.Rn[j * BM + l] = c * hj + s * hj1;
        st.Rn[(j + 1) * BM + l] = -s * hj + c * hj1;
      }
    }
    if (lane < M) {  // columns j, j+1 of Tn
      const double gj = st.Tn[lane * BM + j], gj1 = st.Tn[lane * BM + j + 1];
      st.Tn[lane * BM + j] = c * gj + s * gj1;
      st.Tn[lane * BM + j + 1] = -s * gj + c * gj1;
    }
    __syncwarp();
    if (lane < M) {  // rows j, j+1 of Tn
      const double gj = st.Tn[j * BM + lane], gj1 = st.Tn[(j + 1) * BM + lane];
      st.Tn[j * BM + lane] = c * gj + s * gj1;
      st.Tn[(j + 1) * BM + lane] = -s * gj + c * gj1;
    }
    if (lane == 0) st.Rn[(j + 1) * BM + j] = 0.0;
    const double sj1 = st.sig[j + 1];
    double k1, k2, sout, type;
    if (fabs(c) >= fabs(s)) {
      k1 = s * sj1 / (c * tau);
      k2 = -s * tau / (c * sj1);
      sout = c * tau;
      tau = c * sj1;
      type = 1.0;
    } else {
      k1 = c * tau / (s * sj1);
      k2 = -c * sj1 / (s * tau);
      sout = s * sj1;
      tau = -s * tau;
      type = 0.0;
    }
    if (lane == 0) {
      st.rot[4 * j] = k1;
      st.rot[4 * j + 1] = k2;
      st.rot[4 * j + 2] = type;
      st.rot[4 * j + 3] = sout;
    }
    __syncwarp();
  }
  for (int l = lane; l < M; l += 32) st.Rn[(M - 1) * BM + l] = 0.0;
  for (int i = lane; i < BM * BM; i += 32) {
    const int j = i / BM, l = i % BM;
    double v = 0.0;
    if (j == l && j < M - 1) v = 1.0;
    else if (l < j && j <= M - 3) v = st.Tn[i];
    st.Tn[i] = v;
  }
  if (lane == 0) st.pend = 1;
  __syncwarp();
}

// Warp 0: finish an add (new diagonal, breakdown test, gamma).
__device__ void finalize_b(SState &st, int m, int k, double rho, double vf, double vscale,
                           int head_new, double bd_tol, int lane) {
  const bool bd = !(rho > 0.0) || !isfinite(rho) || rho <= bd_tol * sqrt(st.dfn2);
  if (bd) {
    for (int j = lane; j < BM; j += 32) st.gphys[j] = 0.0;
    if (lane == 0) {
      st.c = 0;
      st.head = 0;
      st.pend = 0;
      st.restarts++;
    }
    __syncwarp();
  } else {
    for (int l = lane; l < m; l += 32) st.R[k * BM + l] = 0.0;
    __syncwarp();
    for (int j = lane; j < k; j += 32) st.R[j * BM + k] = st.rcol[j];
    for (int l = lane; l < m; l += 32) st.T[k * BM + l] = (l == k) ? 1.0 : 0.0;
    if (lane == 0) {
      st.R[k * BM + k] = rho;
      st.sig[k] = 1.0 / (rho * vscale);
      st.rhs[k] = vf / rho;
    }
    __syncwarp();
    // R gamma = rhs by columns: lane j holds rhs_j minus the terms of the
    // unknowns found so far.
    double sj = (lane <= k) ? st.rhs[lane] : 0.0;
    const double inv = (lane <= k) ? 1.0 / st.R[lane * BM + lane] : 0.0;  // in parallel
    for (int l = k; l >= 0; --l) {
      const double gl = __shfl_sync(0xffffffffu, sj * inv, l);
      if (lane < l) sj -= st.R[lane * BM + l] * gl;
      if (lane == l) st.gam[l] = gl;
    }
    for (int j = lane; j < BM; j += 32) st.gphys[j] = 0.0;
    __syncwarp();
    if (lane <= k) st.gphys[(head_new + lane) % m] = st.gam[lane];
    if (lane == 0) {
      st.c = k + 1;
      st.head = head_new;
    }
    __syncwarp();
  }
  if (st.c == m && st.pend == 0) prepare_delete_b(st, m, lane);
}

// MB: history-depth bucket (m <= MB) -- sizes the per-thread accumulators.
template <int NT, int MB>
__global__ void __launch_bounds__(NT, NT <= 128 ? 4 : (NT <= 256 ? 2 : 1)) batch_kernel(BArgs a) {
  constexpr int ND = 3 + 3 * MB;
  __shared__ SState st;
  __shared__ float2 wbuf[(NT / 32) * BNDOT];
  __shared__ float cfr[4 * BM], cfc[2 * BM], cfg[2 * BM], cfv[2];
  __shared__ float2 exptab[aa::EXP_TAB];
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = a.m;
  // staged operands: sd[stage][vector][thread] (FP64), sq[stage][column][thread] (FP32)
  double *const sd = (double *)dsm;
  float *const sq = (float *)(sd + 2 * 4 * NT);
  auto SD = [&](int sg, int v) -> double & { return sd[(sg * 4 + v) * NT + tid]; };
  auto SQ = [&](int sg, int jj) -> float & { return sq[(sg * MB + jj) * NT + tid]; };
  aa::exp_table_init(exptab);

  for (;;) {
    if (tid == 0) st.solve = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int si = st.solve;
    if (si >= a.count) return;
    const Solve S = a.solves[si];
    if (tid == 0) a.res[S.orig].t0 = global_ns();
    const int s = S.s;
    const int64_t n = (int64_t)s * s, off = S.off;
    const double h = 1.0 / (double)(s + 1), h2 = h * h, lam = S.lambda;
    if (tid == 0) {
      st.c = 0;
      st.head = 0;
      st.pend = 0;
      st.done = 0;
      st.status = 1;
      st.restarts = 0;
      st.it = 0;
      st.fallback = 0;
      st.scale = S.scale;
      for (int i = 0; i < BM * BM; ++i) st.R[i] = st.T[i] = 0.0;
    }
    __syncthreads();
    double *Xc = a.X0 + off, *Xn = a.X1 + off;
    double *GP = a.GP + off, *FP = a.FP + off, *DF = a.DF + off;
    const double *src = a.src ? a.src + off : nullptr;
    int it = 0;
    for (;; ++it) {
      const int c = st.c;
      const bool del = (it > 0) && (c == m);
      const int k = (it == 0) ? 0 : (del ? m - 1 : c);
      const int head_new = del ? (st.head + 1) % m : st.head;
      const int dg_slot = del ? st.head : (st.head + c) % m;
      // ---- pass A: G, differences, rotation, first dot block
      if (del) {
        for (int j = tid; j < m - 1; j += NT) {
          const F2 k1 = aa::d2f2(st.rot[4 * j]), k2 = aa::d2f2(st.rot[4 * j + 1]);
          cfr[4 * j] = k1.h;
          cfr[4 * j + 1] = k1.l;
          cfr[4 * j + 2] = k2.h;
          cfr[4 * j + 3] = k2.l;
        }
        __syncthreads();
      }
      float aS[ND], aC[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) aS[d] = aC[d] = 0.f;
      auto stageA = [&](int rr, int sg) {
        if (rr < (int)n) {
          cp_async8(&SD(sg, 0), Xc + rr);
          if (src) cp_async8(&SD(sg, 3), src + rr);
          if (it > 0) {
            cp_async8(&SD(sg, 1), FP + rr);
            cp_async8(&SD(sg, 2), GP + rr);
#pragma unroll
            for (int jj = 0; jj < MB; ++jj)
              if (jj < c) cp_async4(&SQ(sg, jj), a.Q + (int64_t)jj * a.N + off + rr);
          }
        }
        cp_async_commit();
      };
      stageA(tid, 0);
      int sgA = 0;
      // grid coordinates of row r = j s + i, advanced by NT rows per step
      // without a division per row
      int j = tid / s, i = tid - (tid / s) * s;
      const int jstep = NT / s, istep = NT - (NT / s) * s;
      for (int r = tid; r < (int)n; r += NT, sgA ^= 1) {
        if (r != tid) {
          i += istep;
          j += jstep;
          if (i >= s) {
            i -= s;
            ++j;
          }
        }
        stageA(r + NT, sgA ^ 1);
        prefetch_rows(lane, r - lane + PF * NT, n, a.Q + off, a.N, (it == 0) ? 0 : c, Xc, FP, GP, src);
        cp_async_wait<1>();
        const double x = SD(sgA, 0);
        const double w = i > 0 ? Xc[r - 1] : 0.0;
        const double e = i < s - 1 ? Xc[r + 1] : 0.0;
        const double so = j > 0 ? Xc[r - s] : 0.0;
        const double no = j < s - 1 ? Xc[r + s] : 0.0;
        const double rhs = lam * aa::exp_df(x, exptab) + (src ? SD(sgA, 3) : 0.0);
        const double g = ((w + e) + (so + no) + h2 * rhs) * 0.25;
        const double f = g - x;
        const F2 f2 = aa::d2f2(f);
        float p, q;
        aa::prod_ff(f2, f2, p, q);
        aa::acc_add(aS[0], aC[0], p, q);
        if (it == 0) {
          FP[r] = f;
          GP[r] = g;
          continue;
        }
        const double df = f - SD(sgA, 1), dg = g - SD(sgA, 2);
        a.DG[(int64_t)dg_slot * a.N + off + r] = aa::d2f_rn(dg);
        DF[r] = df;
        FP[r] = f;
        GP[r] = g;
        const F2 d2 = aa::d2f2(df);
        aa::prod_ff(d2, d2, p, q);
        aa::acc_add(aS[1], aC[1], p, q);
        aa::prod_ff(d2, f2, p, q);
        aa::acc_add(aS[2], aC[2], p, q);
        if (k == 0) a.Q[off + r] = aa::d2f_rn(df);
        float qv[MB];
#pragma unroll
        for (int jj = 0; jj < MB; ++jj)
          if (jj < c) qv[jj] = SQ(sgA, jj);
        if (del) {
          // the scaled rotations in FP32, two multiply-adds each: the two
          // forms differ in which of (carry w, stored column u) meets which
          // multiplier, out = b + k1 a, carry = a + k2 b with (a, b) = (u, w)
          // when |c| >= |s| and (w, u) otherwise
          float wv = qv[0];
#pragma unroll
          for (int jj = 0; jj < MB - 1; ++jj) {
            if (jj < m - 1) {
              const float u = qv[jj + 1];
              const bool ty = __double_as_longlong(st.rot[4 * jj + 2]) != 0;
              const float pa = ty ? u : wv, pb = ty ? wv : u;
              const float o = __fmaf_rn(cfr[4 * jj], pa, pb);
              wv = __fmaf_rn(cfr[4 * jj + 2], pb, pa);
              qv[jj] = o;
              a.Q[(int64_t)jj * a.N + off + r] = o;
            }
          }
        }
        // Q'^T f (rhs), Q'^T df (R column), Q'^T q'_{k-1} (delayed T row)
#pragma unroll
        for (int jj = 0; jj < MB; ++jj)
          if (jj < k) {
            aa::prod_f(f2, qv[jj], p, q);
            aa::acc_add(aS[3 + jj], aC[3 + jj], p, q);
            aa::prod_f(d2, qv[jj], p, q);
            aa::acc_add(aS[3 + MB + jj], aC[3 + MB + jj], p, q);
            if (jj + 1 < k) {
              p = __fmul_rn(qv[jj], qv[k - 1]);
              q = __fmaf_rn(qv[jj], qv[k - 1], -p);
              aa::acc_add(aS[3 + 2 * MB + jj], aC[3 + 2 * MB + jj], p, q);
            }
          }
      }
      // slots: 0 ||f||^2, 1 ||df||^2, 2 df.f, 3+j q_j.f, 3+MB+j q_j.df, 3+2MB+j q_j.q_{k-1}
      cp_async_wait<0>();
      block_reduce_df<NT, ND>(aS, aC, (it == 0) ? 1 : 3 + 2 * MB + (k > 1 ? k - 1 : 0), wbuf, st);
      // ---- warp 0: stop test, R column, T row, projection coefficients
      if (warp == 0) {
        const double fn2 = st.red[0];
        const double resid = sqrt(fn2) / (st.scale > 0 ? st.scale : 1.0);
        if (lane == 0) {
          if (it == 0 && a.warm && !st.fallback && !(resid < 1.0)) {
            // the warm start is worse than x_0 = 0: restart from zero
            st.fallback = 1;
          } else if (!isfinite(fn2)) {
            st.done = 1;
            st.status = AA_ENONFINITE;
          } else if (resid < a.tol || st.scale == 0.0) {
            st.done = 1;
            st.status = 0;
          } else if (it >= a.max_iters) {
            st.done = 1;
            st.status = 1;
          }
          a.res[S.orig].iters = it;
          a.res[S.orig].resid = resid;
          a.res[S.orig].status = st.status;
          a.res[S.orig].fallback = st.fallback ? 1 : 0;
          if (st.done) a.res[S.orig].t1 = global_ns();
        }
        __syncwarp();
        if (!st.done && it > 0) {
          if (del) {
            for (int i = lane; i < BM * BM; i += 32) {
              const int jj = i / BM, ll = i % BM;
              st.R[i] = (jj < k && ll < k) ? st.Rn[i] : 0.0;
              st.T[i] = st.Tn[i];
            }
            for (int jj = lane; jj < k; jj += 32) st.sig[jj] = st.rot[4 * jj + 3];
            if (lane == 0) st.pend = 0;
            __syncwarp();
          }
          if (lane == 0) {
            st.dfn2 = st.red[1];
            st.vscale = st.dfn2 > 0.0 ? 1.0 / sqrt(st.dfn2) : 1.0;
          }
          for (int jj = lane; jj < k; jj += 32) st.rhs[jj] = st.sig[jj] * st.red[3 + jj];
          if (k > 0) {
            // the delayed T row of column k-1, then the R column r = T^{-1} (Q^T df)
            // by forward substitution with one lane per row
            for (int l = lane; l < BM; l += 32)
              st.T[(k - 1) * BM + l] = (l + 1 < k) ? st.sig[l] * st.sig[k - 1] * st.red[3 + 2 * MB + l]
                                                   : ((l == k - 1) ? 1.0 : 0.0);
            __syncwarp();
            double v = (lane < k) ? st.sig[lane] * st.red[3 + MB + lane] : 0.0;
            for (int l = 0; l + 1 < k; ++l) {
              const double rl = __shfl_sync(0xffffffffu, v, l);
              if (lane > l && lane < k) v -= st.T[lane * BM + l] * rl;
            }
            if (lane < k) {
              st.rcol[lane] = v;
              st.coef[lane] = st.sig[lane] * v;
            }
          }
        }
        __syncwarp();
        if (!st.done && it > 0 && k == 0)
          finalize_b(st, m, 0, sqrt(st.red[1]), st.red[2], 1.0, head_new, a.breakdown_tol, lane);
      }
      __syncthreads();
      if (st.done) break;
      if (it == 0 && st.fallback == 1) {
        for (int64_t r = tid; r < n; r += NT) Xc[r] = 0.0;
        if (tid == 0) st.fallback = 2;
        __syncthreads();
        it = -1;
        continue;
      }
      if (it > 0 && k > 0) {
        // ---- projection pass: v = Delta f - Q r, new column, ||v||, v.f
        for (int jj = tid; jj < k; jj += NT) {
          const F2 cc = aa::d2f2(-st.coef[jj]);
          cfc[2 * jj] = cc.h;
          cfc[2 * jj + 1] = cc.l;
        }
        if (tid == 0) {
          const F2 vs = aa::d2f2(st.vscale);
          cfv[0] = vs.h;
          cfv[1] = vs.l;
        }
        __syncthreads();
        float vS[2] = {0.f, 0.f}, vC[2] = {0.f, 0.f};
        auto stageP = [&](int64_t rr, int sg) {
          if (rr < n) {
            cp_async8(&SD(sg, 0), DF + rr);
            cp_async8(&SD(sg, 1), FP + rr);
#pragma unroll
            for (int jj = 0; jj < MB; ++jj)
              if (jj < k) cp_async4(&SQ(sg, jj), a.Q + (int64_t)jj * a.N + off + rr);
          }
          cp_async_commit();
        };
        stageP(tid, 0);
        int sgP = 0;
        for (int64_t r = tid; r < n; r += NT, sgP ^= 1) {
          stageP(r + NT, sgP ^ 1);
          prefetch_rows(lane, r - lane + PF * NT, n, a.Q + off, a.N, k, DF, FP, nullptr, nullptr);
          cp_async_wait<1>();
          // v = Delta f - Q r: FP32 chains of the coefficients' heads and
          // tails over the stored columns, added to Delta f in FP64
          float s0 = 0.f, s1 = 0.f, sl = 0.f;
#pragma unroll
          for (int jj = 0; jj < MB; ++jj)
            if (jj < k) {
              const float qj = SQ(sgP, jj);
              if (jj & 1) s1 = __fmaf_rn(cfc[2 * jj], qj, s1);
              else s0 = __fmaf_rn(cfc[2 * jj], qj, s0);
              sl = __fmaf_rn(cfc[2 * jj + 1], qj, sl);
            }
          const F2 acc = aa::d2f2(SD(sgP, 0) + (aa::f2d(__fadd_rn(s0, s1)) + aa::f2d(sl)));
          float p, q;
          aa::prod_ff(acc, F2{cfv[0], cfv[1]}, p, q);
          a.Q[(int64_t)k * a.N + off + r] = __fadd_rn(p, q);
          aa::prod_ff(acc, acc, p, q);
          aa::acc_add(vS[0], vC[0], p, q);
          aa::prod_ff(acc, aa::d2f2(SD(sgP, 1)), p, q);
          aa::acc_add(vS[1], vC[1], p, q);
        }
        cp_async_wait<0>();
        block_reduce_df<NT, 2>(vS, vC, 2, wbuf, st);
        if (warp == 0)
          finalize_b(st, m, k, sqrt(st.red[0]), st.red[1], st.vscale, head_new, a.breakdown_tol,
                     lane);
        __syncthreads();
      }
      // ---- update pass: x_{i+1} = G(x_i) - dG gamma
      const int ng = (it == 0) ? 0 : st.c;
      for (int jj = tid; jj < BM; jj += NT) {
        const F2 gg = aa::d2f2(-st.gphys[jj]);
        cfg[2 * jj] = gg.h;
        cfg[2 * jj + 1] = gg.l;
      }
      if (tid == 0) {
        unsigned mk = 0;
        for (int jj = 0; jj < m; ++jj)
          if (st.gphys[jj] != 0.0) mk |= 1u << jj;
        st.gmask = mk;
      }
      __syncthreads();
      const unsigned gmask = st.gmask;
      auto stageU = [&](int64_t rr, int sg) {
        if (rr < n) {
          cp_async8(&SD(sg, 0), GP + rr);
#pragma unroll
          for (int jj = 0; jj < MB; ++jj)
            if ((gmask >> jj) & 1u) cp_async4(&SQ(sg, jj), a.DG + (int64_t)jj * a.N + off + rr);
        }
        cp_async_commit();
      };
      stageU(tid, 0);
      int sgU = 0;
      for (int64_t r = tid; r < n; r += NT, sgU ^= 1) {
        stageU(r + NT, sgU ^ 1);
        prefetch_rows(lane, r - lane + PF * NT, n, a.DG + off, a.N, ng, GP, nullptr, nullptr, nullptr);
        cp_async_wait<1>();
        if (ng == 0) {
          Xn[r] = SD(sgU, 0);
          continue;
        }
        // x_{i+1} = G(x_i) - dG gamma: FP32 chains (heads, tails), added in FP64
        float s0 = 0.f, s1 = 0.f, sl = 0.f;
#pragma unroll
        for (int jj = 0; jj < MB; ++jj)
          if ((gmask >> jj) & 1u) {
            const float dj = SQ(sgU, jj);
            if (jj & 1) s1 = __fmaf_rn(cfg[2 * jj], dj, s1);
            else s0 = __fmaf_rn(cfg[2 * jj], dj, s0);
            sl = __fmaf_rn(cfg[2 * jj + 1], dj, sl);
          }
        Xn[r] = SD(sgU, 0) + (aa::f2d(__fadd_rn(s0, s1)) + aa::f2d(sl));
      }
      cp_async_wait<0>();
      __syncthreads();
      double *tmp = Xc;
      Xc = Xn;
      Xn = tmp;
    }
    // leave the returned iterate in X0
    if (Xc != a.X0 + off)
      for (int64_t r = tid; r < n; r += NT) a.X0[off + r] = Xc[r];
    __syncthreads();
  }
}

}  // namespace

struct aa_batch {
  int count, m;
  int64_t N;
  std::vector<Solve> hsolves;
  std::vector<int64_t> side;
  Solve *dsolves;
  Result *dres;
  double *X0, *X1, *GP, *FP, *DF, *src, *Xinit;
  float *Q, *DG;
  unsigned *queue;
  double tol, bd_tol;
  int max_iters, block, ctas_per_sm;
  cudaGraphExec_t gexec;
  cudaGraph_t graph;
  cudaStream_t gstream;
};

static int64_t round_up64(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

extern "C" int aa_batch_create(const aa_batch_desc *d, aa_batch **out) {
  if (!d || !out || d->count < 1 || !d->side || !d->lambda) return AA_EINVAL;
  if (d->m < 1 || d->m > BM) return AA_EINVAL;
  *out = nullptr;
  aa_batch *b = new (std::nothrow) aa_batch();
  if (!b) return AA_ENOMEM;
  b->count = d->count;
  b->m = d->m;
  b->tol = d->tol > 0 ? d->tol : 1e-8;
  b->bd_tol = 1e-14;
  b->max_iters = d->max_iters > 0 ? d->max_iters : 100000;
  b->block = d->block;
  b->ctas_per_sm = d->ctas_per_sm;
  // largest solves first
  std::vector<int> order(d->count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return d->side[x] > d->side[y]; });
  int64_t off = 0;
  b->hsolves.resize(d->count);
  for (int i = 0; i < d->count; ++i) {
    const int o = order[i];
    if (d->side[o] < 1 || d->side[o] > 46340) {
      delete b;
      return AA_EINVAL;
    }
    Solve S;
    S.off = off;
    S.s = (int32_t)d->side[o];
    S.orig = o;
    S.lambda = d->lambda[o];
    S.scale = 0.0;
    b->hsolves[i] = S;
    off += round_up64((int64_t)S.s * S.s, 64);
  }
  b->N = off;
  const size_t nd = (size_t)b->N * sizeof(double), nf = (size_t)b->N * sizeof(float);
  bool ok = cudaMalloc(&b->X0, nd) == cudaSuccess && cudaMalloc(&b->X1, nd) == cudaSuccess &&
            cudaMalloc(&b->GP, nd) == cudaSuccess && cudaMalloc(&b->FP, nd) == cudaSuccess &&
            cudaMalloc(&b->DF, nd) == cudaSuccess &&
            cudaMalloc(&b->Q, nf * b->m) == cudaSuccess &&
            cudaMalloc(&b->DG, nf * b->m) == cudaSuccess &&
            cudaMalloc(&b->dsolves, sizeof(Solve) * b->count) == cudaSuccess &&
            cudaMalloc(&b->dres, sizeof(Result) * b->count) == cudaSuccess &&
            cudaMalloc(&b->queue, sizeof(unsigned)) == cudaSuccess;
  // stopping scale ||G(0)||: at u = 0 every neighbour is 0 and e^0 = 1, so
  // G(0)_p = h^2 (lambda + src_p) / 4.
  {
    std::vector<int64_t> corig(d->count);
    int64_t so = 0;
    for (int i = 0; i < d->count; ++i) {
      corig[i] = so;
      so += d->side[i] * d->side[i];
    }
    for (Solve &S : b->hsolves) {
      const double h = 1.0 / (double)(S.s + 1);
      const int64_t n = (int64_t)S.s * S.s;
      double acc = 0.0;
      for (int64_t p = 0; p < n; ++p) {
        const double v = S.lambda + (d->src_host ? d->src_host[corig[S.orig] + p] : 0.0);
        acc += v * v;
      }
      S.scale = h * h / 4.0 * sqrt(acc);
    }
  }
  if (ok && d->src_host) {
    ok = cudaMalloc(&b->src, nd) == cudaSuccess;
    if (ok) {
      std::vector<double> hs(b->N, 0.0);
      int64_t so = 0;  // src_host is in the caller's order, concatenated
      std::vector<int64_t> corig(d->count);
      for (int i = 0; i < d->count; ++i) {
        corig[i] = so;
        so += d->side[i] * d->side[i];
      }
      for (const Solve &S : b->hsolves)
        memcpy(&hs[S.off], d->src_host + corig[S.orig], sizeof(double) * (size_t)S.s * S.s);
      ok = cudaMemcpy(b->src, hs.data(), nd, cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (ok)
    ok = cudaMemcpy(b->dsolves, b->hsolves.data(), sizeof(Solve) * b->count,
                    cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    aa_batch_destroy(b);
    return AA_ENOMEM;
  }
  *out = b;
  return AA_OK;
}

extern "C" void aa_batch_destroy(aa_batch *b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->X0);
  cudaFree(b->X1);
  cudaFree(b->GP);
  cudaFree(b->FP);
  cudaFree(b->DF);
  cudaFree(b->Q);
  cudaFree(b->DG);
  cudaFree(b->src);
  cudaFree(b->Xinit);
  cudaFree(b->dsolves);
  cudaFree(b->dres);
  cudaFree(b->queue);
  delete b;
}

template <int NT, int MB>
static cudaError_t launch_mb(const BArgs &a, int grid, cudaStream_t s) {
  batch_kernel<NT, MB><<<grid, NT, stage_bytes(NT, MB), s>>>(a);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_batch(const BArgs &a, int grid, cudaStream_t s) {
  if (a.m <= 4) return launch_mb<NT, 4>(a, grid, s);
  if (a.m <= 8) return launch_mb<NT, 8>(a, grid, s);
  if (a.m <= 10) return launch_mb<NT, 10>(a, grid, s);
  if (a.m <= 12) return launch_mb<NT, 12>(a, grid, s);
  return launch_mb<NT, 16>(a, grid, s);
}

// The staging buffer is dynamic shared memory (up to 96 KB at 512 threads):
// raise every instance's limit once, outside any stream capture.
template <int NT>
static cudaError_t smem_attr_nt() {
  cudaError_t e = cudaSuccess;
  const int mbs[5] = {4, 8, 10, 12, 16};
  for (int mb : mbs) {
    const void *f = mb == 4    ? (const void *)batch_kernel<NT, 4>
                    : mb == 8  ? (const void *)batch_kernel<NT, 8>
                    : mb == 10 ? (const void *)batch_kernel<NT, 10>
                    : mb == 12 ? (const void *)batch_kernel<NT, 12>
                               : (const void *)batch_kernel<NT, 16>;
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)stage_bytes(NT, mb));
    if (r != cudaSuccess) e = r;
  }
  return e;
}

static cudaError_t smem_attrs() {
  static bool done = false;  // per process; the attribute holds for every device context
  if (done) return cudaSuccess;
  cudaError_t e = smem_attr_nt<128>();
  if (e == cudaSuccess) e = smem_attr_nt<256>();
  if (e == cudaSuccess) e = smem_attr_nt<512>();
  if (e == cudaSuccess) done = true;
  return e;
}

static cudaError_t enqueue(aa_batch *b, int block, int cps, cudaStream_t s) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  BArgs a;
  a.solves = b->dsolves;
  a.res = b->dres;
  a.count = b->count;
  a.m = b->m;
  a.max_iters = b->max_iters;
  a.tol = b->tol;
  a.breakdown_tol = b->bd_tol;
  a.X0 = b->X0;
  a.X1 = b->X1;
  a.GP = b->GP;
  a.FP = b->FP;
  a.DF = b->DF;
  a.Q = b->Q;
  a.DG = b->DG;
  a.N = b->N;
  a.src = b->src;
  a.warm = b->Xinit != nullptr;
  a.queue = b->queue;
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = b->Xinit ? cudaMemcpyAsync(b->X0, b->Xinit, (size_t)b->N * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s)
                 : cudaMemsetAsync(b->X0, 0, (size_t)b->N * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const int grid = nsm * (cps > 0 ? cps : 1);
  switch (block) {
    case 128: return launch_batch<128>(a, grid, s);
    case 512: return launch_batch<512>(a, grid, s);
    default: return launch_batch<256>(a, grid, s);
  }
}

extern "C" int aa_batch_solve(aa_batch *b, int block, int ctas_per_sm, void *stream,
                              double *ms_out) {
  if (!b) return AA_EINVAL;
  if (block != 128 && block != 256 && block != 512) block = 256;
  if (ctas_per_sm < 1 || ctas_per_sm > 4) ctas_per_sm = 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (smem_attrs() != cudaSuccess) {
    cudaGetLastError();
    return AA_ECUDA;
  }
  // The whole batch is one persistent kernel; it is captured once per
  // (block, ctas_per_sm) into a CUDA graph and replayed.
  if (!b->gexec || b->block != block || b->ctas_per_sm != ctas_per_sm) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return AA_ECUDA;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(b, block, ctas_per_sm, cs);
      e = cudaStreamEndCapture(cs, &b->graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return AA_ECUDA;
    }
    b->block = block;
    b->ctas_per_sm = ctas_per_sm;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t e = cudaGraphLaunch(b->gexec, s);
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_out) *ms_out = ms;
  return e == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_batch_results(aa_batch *b, int32_t *iters, double *resid, int32_t *status) {
  if (!b) return AA_EINVAL;
  std::vector<Result> r(b->count);
  if (cudaMemcpy(r.data(), b->dres, sizeof(Result) * b->count, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return AA_ECUDA;
  for (int i = 0; i < b->count; ++i) {
    if (iters) iters[i] = r[i].iters;
    if (resid) resid[i] = r[i].resid;
    if (status) status[i] = r[i].status;
  }
  return AA_OK;
}

extern "C" int aa_batch_fallbacks(aa_batch *b, int32_t *fallback) {
  if (!b || !fallback) return AA_EINVAL;
  std::vector<Result> r(b->count);
  if (cudaMemcpy(r.data(), b->dres, sizeof(Result) * b->count, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return AA_ECUDA;
  for (int i = 0; i < b->count; ++i) fallback[i] = r[i].fallback;
  return AA_OK;
}

extern "C" int aa_batch_solution(aa_batch *b, int idx, double *x_host) {
  if (!b || idx < 0 || idx >= b->count || !x_host) return AA_EINVAL;
  for (const Solve &S : b->hsolves)
    if (S.orig == idx) {
      if (cudaMemcpy(x_host, b->X0 + S.off, sizeof(double) * (size_t)S.s * S.s,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
        return AA_ECUDA;
      return AA_OK;
    }
  return AA_EINVAL;
}

extern "C" int aa_batch_times(aa_batch *b, double *start_ms, double *end_ms) {
  if (!b || (!start_ms && !end_ms)) return AA_EINVAL;
  std::vector<Result> r(b->count);
  if (cudaMemcpy(r.data(), b->dres, sizeof(Result) * b->count, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return AA_ECUDA;
  uint64_t t_min = UINT64_MAX;
  for (const Result &x : r) t_min = std::min(t_min, x.t0);
  for (int i = 0; i < b->count; ++i) {
    if (start_ms) start_ms[i] = (double)(r[i].t0 - t_min) * 1e-6;
    if (end_ms) end_ms[i] = (double)(r[i].t1 - t_min) * 1e-6;
  }
  return AA_OK;
}

extern "C" int64_t aa_batch_rows(const aa_batch *b) { return b ? b->N : 0; }

extern "C" int aa_batch_set_max_iters(aa_batch *b, int max_iters) {
  if (!b || max_iters < 1) return AA_EINVAL;
  if (b->max_iters != max_iters) {
    b->max_iters = max_iters;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
  }
  return AA_OK;
}

namespace {
__global__ void exp_kernel(int64_t n, const double *__restrict__ u, double *__restrict__ out) {
  __shared__ float2 tab[aa::EXP_TAB];
  aa::exp_table_init(tab);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = aa::exp_df(u[i], tab);
}
}  // namespace

extern "C" int aa_exp_fp32pipe(int64_t n, const double *u, double *out, void *stream) {
  if (n < 1 || !u || !out) return AA_EINVAL;
  const int64_t g = (n + 255) / 256;
  exp_kernel<<<(int)(g > 4096 ? 4096 : g), 256, 0, (cudaStream_t)stream>>>(n, u, out);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_batch_set_x0(aa_batch *b, const double *x0_host) {
  if (!b) return AA_EINVAL;
  if (!x0_host) {  // back to x_0 = 0
    cudaFree(b->Xinit);
    b->Xinit = nullptr;
  } else {
    if (!b->Xinit && cudaMalloc(&b->Xinit, (size_t)b->N * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return AA_ENOMEM;
    }
    std::vector<double> hx(b->N, 0.0);
    std::vector<int64_t> corig(b->count);
    int64_t so = 0;
    std::vector<int64_t> side_orig(b->count);
    for (const Solve &S : b->hsolves) side_orig[S.orig] = S.s;
    for (int i = 0; i < b->count; ++i) {
      corig[i] = so;
      so += side_orig[i] * side_orig[i];
    }
    for (const Solve &S : b->hsolves)
      memcpy(&hx[S.off], x0_host + corig[S.orig], sizeof(double) * (size_t)S.s * S.s);
    if (cudaMemcpy(b->Xinit, hx.data(), (size_t)b->N * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return AA_ECUDA;
  }
  // the captured graph embeds the x_0 copy: capture again on the next solve
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  return AA_OK;
}
