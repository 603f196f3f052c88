#pragma once
// aa_passes.cuh -- streaming-pass kernels of the low-synchronization
// Anderson-acceleration hot path for sm_103a.
//
// One kernel template serves every pass.  A persistent grid walks row tiles
// of TR rows.  For each tile one thread issues bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) of the pass's columns into a
// shared-memory stage; STAGES stages keep the next tile's copies in flight
// while the current tile is processed.  The per-row program runs one thread
// per row and writes its outputs straight to global memory with coalesced
// stores; the dot phase then has each warp accumulate a subset of the
// pass's dot products over the tile.  At the end every CTA writes its
// per-dot partial sums to a slot array; the last CTA to take a ticket sums
// the slots in CTA order -- a deterministic grid-wide reduction, the
// single-GPU form of the paper's global reduction -- and runs the small
// m x m part of the algorithm (R, T, gamma) in the same launch.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "aa_common.h"
#include "aa_df.cuh"



namespace aa {

// Error codes raised on the device (mirror of aa.h).
constexpr int DEV_ENONFINITE = -5;
constexpr int DEV_ETIMEOUT = -6;

// ------------------------------------------------------------ conversions

template <class QT> __device__ __forceinline__ double to_d(QT v);
template <> __device__ __forceinline__ double to_d<double>(double v) { return v; }
// float/bf16 <-> double through integer operations (the hardware conversion
// instructions run on the scarce FP64 pipe of this part).
template <> __device__ __forceinline__ double to_d<float>(float v) { return f2d(v); }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) {
  return f2d(__bfloat162float(v));
}
template <class QT> __device__ __forceinline__ QT from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return d2f_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn(d2f_rn(v));
}
template <class QT> __device__ __forceinline__ float q2f(QT v);
template <> __device__ __forceinline__ float q2f<float>(float v) { return v; }
template <> __device__ __forceinline__ float q2f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float q2f<double>(double v) { return (float)v; }  // not called: FP64 paths split with d2f2
template <class QT> __device__ __forceinline__ QT f2q(float v);
template <> __device__ __forceinline__ float f2q<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 f2q<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ double f2q<double>(float v) { return (double)v; }  // not called on FP64 paths

// ------------------------------------------------- mbarrier / bulk copies

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  (void)state;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, "
      "0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up once a second has passed on the device's global
// timer (checked every 64 tries; try_wait itself suspends only for a short,
// system-defined time), with an iteration cap as a second bound.  On expiry
// the pass records DEV_ETIMEOUT and the caller stops issuing work.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > 1000000000ull) return false;
    if (i > 32) __nanosleep(256);
  }
  return false;
}

// ------------------------------------------------------------- tile access

// Stage layout: the FP64 columns 0..qbase-1 first (TR doubles each; the
// FP32-pipe forms overwrite them in place with (hi, lo) float pairs), then
// the history columns at their storage width (TR elements each), so that an
// FP32 or BF16 history stage takes a half or a quarter of the FP64 space.
struct Stage {
  unsigned char *base;
  int qbase;
  __device__ __forceinline__ double *d(int c) const { return (double *)(base + c * (TR * 8)); }
  template <class QT>
  __device__ __forceinline__ QT *q(int c) const {
    if constexpr (sizeof(QT) == 8) return (QT *)(base + c * (TR * 8));
    else return (QT *)(base + qbase * (TR * 8) + (c - qbase) * (int)(TR * sizeof(QT)));
  }
  // An FP64 column after it was split in place into (hi, lo) floats, laid
  // out by row pairs: rows 2i and 2i+1 as (hi_2i, hi_2i+1, lo_2i, lo_2i+1),
  // so that one 16-byte load gives the two rows' heads and tails as float2s.
  __device__ __forceinline__ float *p(int c) const { return (float *)(base + c * (TR * 8)); }
  __device__ __forceinline__ F2 f2(int c, int r) const {
    const float *q = p(c) + (r >> 1) * 4 + (r & 1);
    return F2{q[0], q[2]};
  }
  __device__ __forceinline__ void put(int c, int r, F2 v) const {
    float *q = p(c) + (r >> 1) * 4 + (r & 1);
    q[0] = v.h;
    q[2] = v.l;
  }
  // rows r, r + 1 (r even): heads in .x/.y of hl[0], tails in hl[1]
  __device__ __forceinline__ float4 pairs2(int c, int r) const {
    return *(const float4 *)(p(c) + (r >> 1) * 4);
  }
};

// History slot j as an output (slots are qstride bytes apart: an address
// computation, not a load of a pointer table from parameter space).
template <class QT>
__device__ __forceinline__ QT *outq(const PassArgs &a, int j) {
  return (QT *)((char *)a.out_q0 + (int64_t)j * a.qstride);
}

template <class QT>
__device__ __forceinline__ int col_esz(const PassArgs &a, int c) {
  return c >= a.qbase ? (int)sizeof(QT) : 8;
}

// Bytes of one stage (see Stage), a multiple of 128.
template <class QT>
__host__ __device__ __forceinline__ size_t stage_size(const PassArgs &a) {
  const size_t b = (size_t)a.qbase * TR * 8 + (size_t)(a.ncol - a.qbase) * TR * sizeof(QT);
  return (b + 127) / 128 * 128;
}

// Issue the bulk copies of tile t into stage st (one thread).  Rows are
// copied in multiples of 8 (16 bytes for the narrowest storage type); the
// remaining < 8 rows of a ragged last tile are loaded by their threads.
template <class QT>
static __device__ void issue_tile(const PassArgs &a, Stage st, int t, uint64_t *bar) {
  const int64_t r0 = (int64_t)t * TR;
  const int rows = (int)min((int64_t)TR, a.n - r0);
  const int rt = rows & ~7;
  uint32_t bytes = 0;
  for (int c = 0; c < a.ncol; ++c) bytes += (uint32_t)(rt * col_esz<QT>(a, c));
  mbar_arrive_expect_tx(bar, bytes);
  if (rt > 0) {
    size_t off = 0;
    for (int c = 0; c < a.ncol; ++c) {
      const int es = col_esz<QT>(a, c);
      const char *src = (const char *)a.col[c] + r0 * es;
      bulk_g2s(st.base + off, src, (uint32_t)(rt * es), bar);
      off += (size_t)TR * es;
    }
  }
}

template <class QT>
__device__ __forceinline__ void load_tail_row(const PassArgs &a, Stage st, int t, int r) {
  const int64_t row = (int64_t)t * TR + r;
  for (int c = 0; c < a.ncol; ++c) {
    if (c >= a.qbase)
      st.q<QT>(c)[r] = ((const QT *)a.col[c])[row];
    else
      st.d(c)[r] = ((const double *)a.col[c])[row];
  }
}

// Rows r and r + 1 (r even) of a stored history column as floats.
template <class QT>
__device__ __forceinline__ float2 q2rows(Stage st, int c, int r);
template <>
__device__ __forceinline__ float2 q2rows<float>(Stage st, int c, int r) {
  return *(const float2 *)(st.q<float>(c) + r);
}
template <>
__device__ __forceinline__ float2 q2rows<__nv_bfloat16>(Stage st, int c, int r) {
  return __bfloat1622float2(*(const __nv_bfloat162 *)(st.q<__nv_bfloat16>(c) + r));
}
template <>
__device__ __forceinline__ float2 q2rows<double>(Stage st, int c, int r) {  // not called
  const double *q = st.q<double>(c) + r;
  return make_float2((float)q[0], (float)q[1]);
}

template <class QT>
__device__ __forceinline__ double ldv(Stage st, int c, int r, bool isq) {
  return isq ? to_d<QT>(st.q<QT>(c)[r]) : st.d(c)[r];
}

// ----------------------------------------------------------- row programs

// Shared coefficient block layout (doubles).
constexpr int CO_ROT = 0;              // 4*(m-1) folded rotation coefficients
constexpr int CO_ROT0 = 4 * MMAX;      // sig_0
constexpr int CO_COEF = 4 * MMAX + 1;  // coef[0..k)
constexpr int CO_COEF2 = 5 * MMAX + 1; // coef2[0..k-1)
constexpr int CO_MISC = 6 * MMAX + 1;  // rcself, vscale
constexpr int CO_SIZE = 6 * MMAX + 4;
// (hi, lo) float copies used by the FP32-pipe programs; projection and update
// coefficients are stored negated.
constexpr int CF_ROT = 0;               // per rotation: k1 (hi, lo), k2 (hi, lo)
constexpr int CF_COEF = 4 * MMAX;       // -coef[j] (hi, lo)
constexpr int CF_COEF2 = 6 * MMAX;      // -coef2[j] (hi, lo)
constexpr int CF_MISC = 8 * MMAX;       // rcself (hi, lo), vscale (hi, lo)
constexpr int CF_SIZE = 8 * MMAX + 4;

template <class QT>
__device__ __forceinline__ void row_program(const PassArgs &a, Stage st, int t, int r,
                                            const double *co) {
  const int64_t row = (int64_t)t * TR + r;
  switch (a.kind) {
    case K_INIT: {
      const double x = st.d(0)[r], g = st.d(1)[r];
      const double f = g - x;
      a.out_f[row] = f;
      a.out_g[row] = g;
      a.out_x[row] = g;
      st.d(0)[r] = f;
      break;
    }
    case K_A: {
      double df;
      if (a.step_mode) {
        const double x = st.d(0)[r], g = st.d(1)[r], gp = st.d(2)[r], fp = st.d(3)[r];
        const double f = g - x;
        df = f - fp;
        const double dg = g - gp;
        ((QT *)a.out_dg)[row] = from_d<QT>(dg);
        a.out_f[row] = f;
        a.out_g[row] = g;
        st.d(0)[r] = f;
        st.d(1)[r] = df;
      } else {
        df = st.d(0)[r];
      }
      a.out_df[row] = df;
      if (a.k == 0) outq<QT>(a, 0)[row] = from_d<QT>(df);
      if (a.del) {
        // QRDelete: sequential Givens rotations of adjacent columns, in the
        // square-root-free scaled form (Gentleman 1973, Hammarling 1974):
        // two multiply-adds per rotation, the scale factors folded into the
        // column scales at the m x m level.  Column j is final once rotation
        // j has been applied; w carries column j+1 (scale tracked on the
        // device state).
        const int qb = a.qbase;
        double w = to_d<QT>(st.q<QT>(qb)[r]);
        for (int j = 0; j < a.m - 1; ++j) {
          const double u = to_d<QT>(st.q<QT>(qb + j + 1)[r]);
          const double *R = co + CO_ROT + 4 * j;
          // The two forms (|c| >= |s| or not; integer test, no FP64 op)
          // differ only in which multiplier goes with which operand and
          // which result is kept: select those, so that exactly two
          // multiply-adds are issued (a branch here may be if-converted
          // into both forms, four multiply-adds).
          const bool ty = __double_as_longlong(R[2]) != 0;
          const double kp = ty ? R[0] : R[1], kq = ty ? R[1] : R[0];
          const double P = fma(kp, u, w);   // w + kp u
          const double Qv = fma(kq, w, u);  // u + kq w
          const double out = ty ? P : Qv;
          w = ty ? Qv : P;
          const QT qs = from_d<QT>(out);
          outq<QT>(a, j)[row] = qs;
          st.q<QT>(qb + j)[r] = qs;
        }
      }
      break;
    }
    case K_PROJ: {
      const int qb = a.qbase;
      double v = st.d(0)[r];
      if (a.orth == O_DCGS2 && (a.flags & 0x100u)) {
        // DCGS-2: correct q_{k-1} against q_0..q_{k-2}, store it, then
        // project v against the corrected factor.
        const int kk = a.k - 1;
        double qn = co[CO_MISC] * to_d<QT>(st.q<QT>(qb + kk)[r]);
        for (int j = 0; j < kk; ++j) qn -= co[CO_COEF2 + j] * to_d<QT>(st.q<QT>(qb + j)[r]);
        const QT qs = from_d<QT>(qn);
        outq<QT>(a, kk)[row] = qs;
        st.q<QT>(qb + kk)[r] = qs;
      }
      for (int j = a.j0; j < a.k; ++j) v -= co[CO_COEF + j] * to_d<QT>(st.q<QT>(qb + j - a.j0)[r]);
      outq<QT>(a, a.k)[row] = from_d<QT>(v * co[CO_MISC + 1]);
      st.d(0)[r] = v;
      break;
    }
    case K_CGS2B: {
      double y = st.d(0)[r];
      for (int j = 0; j < a.k; ++j) y -= co[CO_COEF + j] * to_d<QT>(st.q<QT>(a.qbase + j)[r]);
      a.out_df[row] = y;
      st.d(0)[r] = y;
      break;
    }
    case K_MGS: {
      const double v = st.d(0)[r] - co[CO_COEF + a.jm - 1] * to_d<QT>(st.q<QT>(a.qbase)[r]);
      a.out_df[row] = v;
      st.d(0)[r] = v;
      break;
    }
    case K_UPDATE: {
      double xn = st.d(0)[r];
      for (int i = 0; i < a.ng; ++i) xn -= co[CO_COEF + i] * to_d<QT>(st.q<QT>(a.qbase + i)[r]);
      a.out_x[row] = xn;
      if (a.stop_kind == 1) st.d(1)[r] = xn - st.d(1)[r];
      break;
    }
    default:
      break;
  }
}

// Row programs of the FP32/BF16-history form (MODE 2).  The history columns
// are stored in FP32 or BF16, and the n-space arithmetic on them runs in FP32
// on the FP32 pipe: the QRDelete rotation (two multiply-adds per rotation,
// multipliers rounded to float), the Gram-Schmidt projections v = w - Q c
// (the CGS-2 middle pass and an MGS link alike) and the update
// x = g - dG gamma.  The projection and update coefficients are FP64 and
// enter as (hi, lo) float pairs, each part in its own multiply-add chain
// (lp_chain): a coefficient rounded to float would leave an error along the
// history columns themselves, inside span(Q).  The float multipliers of the
// rotation make each rotated pair orthogonal only to about the float unit
// roundoff u = 2^-24 (adding their tails after a rounded multiply-add would
// round away), and that sets this form's orthogonality loss, about
// u sqrt(m); the storage rounding alone gives random errors, about u / sqrt(n)
// per inner product.  The vectors x, G(x), f, Delta f, v and y stay FP64:
// the residual differences are FP64 adds, and a projection or update sum is
// added to its FP64 vector in FP64.  Dot products stay exact to about 2^-44:
// those whose two operands are FP64 vectors (squared norms, v.f, Delta f.f)
// accumulate row by row in FP64 registers (dv0, dv1 return the row's values
// of FP64 columns 0 and 1 for that); those with a history column run in the
// dot phase on (hi, lo) splits of the FP64 operands, which the row program
// leaves in shared memory for the columns set in `split`.

// sum_j c_j q_j over cnt stored columns q_j = stage column qb + j (row r),
// c_j given as (hi, lo) float pairs at c[2j], c[2j+1]: two FP32 chains of
// the heads (independent, for latency) and one of the tails, returned as an
// FP64 value (converted by integer operations: the hardware float <-> double
// conversions occupy the FP64 pipe, which is the scarce unit on this part).
template <class QT>
__device__ __forceinline__ double lp_chain(Stage st, const float *c, int qb, int cnt, int r) {
  float s0 = 0.f, s1 = 0.f, sl = 0.f;
  int j = 0;
  const QT *qp = st.q<QT>(qb) + r;
#pragma unroll 2
  for (; j + 1 < cnt; j += 2, qp += 2 * TR) {
    const float2 c0 = *(const float2 *)(c + 2 * j), c1 = *(const float2 *)(c + 2 * j + 2);
    const float q0 = q2f<QT>(qp[0]), q1 = q2f<QT>(qp[TR]);
    s0 = __fmaf_rn(c0.x, q0, s0);
    s1 = __fmaf_rn(c1.x, q1, s1);
    sl = __fmaf_rn(c0.y, q0, sl);
    sl = __fmaf_rn(c1.y, q1, sl);
  }
  if (j < cnt) {
    const float2 cc = *(const float2 *)(c + 2 * j);
    const float q0 = q2f<QT>(qp[0]);
    s0 = __fmaf_rn(cc.x, q0, s0);
    sl = __fmaf_rn(cc.y, q0, sl);
  }
  return f2d(__fadd_rn(s0, s1)) + f2d(sl);
}

template <class QT>
__device__ __forceinline__ void row_program_lp(const PassArgs &a, Stage st, int t, int r,
                                               const double *co, const float *cf, uint32_t split,
                                               uint64_t tymask, double &dv0, double &dv1) {
  const int64_t row = (int64_t)t * TR + r;
  switch (a.kind) {
    case K_INIT: {
      const double x = st.d(0)[r], g = st.d(1)[r];
      const double f = g - x;
      a.out_f[row] = f;
      a.out_g[row] = g;
      a.out_x[row] = g;
      dv0 = f;
      break;
    }
    case K_A: {
      double df, f = 0.0;
      if (a.step_mode) {
        const double x = st.d(0)[r], g = st.d(1)[r], gp = st.d(2)[r], fp = st.d(3)[r];
        f = g - x;
        df = f - fp;
        const double dg = g - gp;
        ((QT *)a.out_dg)[row] = f2q<QT>(d2f_rn(dg));
        a.out_f[row] = f;
        a.out_g[row] = g;
        dv0 = f;
        dv1 = df;
        if (split & 1u) st.put(0, r, d2f2(f));
        if (split & 2u) st.put(1, r, d2f2(df));
      } else {
        df = st.d(0)[r];
        dv0 = df;
        if (split & 1u) st.put(0, r, d2f2(df));
      }
      a.out_df[row] = df;
      if (a.k == 0) outq<QT>(a, 0)[row] = f2q<QT>(d2f_rn(df));
      if (a.del) {
        // QRDelete: the scaled Givens rotations of row_program in FP32.  The
        // two forms differ in which of (carry w, stored column u) meets
        // which multiplier: out = b + k1 a, carry = a + k2 b with
        // (a, b) = (u, w) when |c| >= |s| and (w, u) otherwise.
        // (Pointers advanced by one column per rotation; the form of each
        // rotation is bit j of tymask.)
        QT *sq = st.q<QT>(a.qbase) + r;                      // stage column j: sq[j * TR]
        char *gq = (char *)a.out_q0 + row * (int64_t)sizeof(QT);  // slot j: gq + j * qstride
        const float4 *kq = (const float4 *)(cf + CF_ROT);    // k1 (hi, lo), k2 (hi, lo)
        float w = q2f<QT>(sq[0]);
        uint64_t tm = tymask;
#pragma unroll 4
        for (int j = 0; j < a.m - 1; ++j, tm >>= 1) {
          const float u = q2f<QT>(sq[TR]);
          const float4 k = kq[j];
          const bool ty = tm & 1ull;
          const float pa = ty ? u : w, pb = ty ? w : u;
          const QT qs = f2q<QT>(__fmaf_rn(k.x, pa, pb));
          w = __fmaf_rn(k.z, pb, pa);
          *(QT *)gq = qs;
          sq[0] = qs;
          sq += TR;
          gq += a.qstride;
        }
      }
      break;
    }
    case K_PROJ: {
      const int qb = a.qbase;
      if (a.orth == O_DCGS2 && (a.flags & 0x100u)) {
        // DCGS-2: correct q_{k-1} against q_0..q_{k-2}, store it, then
        // project against the corrected factor
        const int kk = a.k - 1;
        const float qk = q2f<QT>(st.q<QT>(qb + kk)[r]);
        float qn = cf[CF_MISC] * qk, ql = cf[CF_MISC + 1] * qk;
        for (int j = 0; j < kk; ++j) {
          const float2 c = *(const float2 *)(cf + CF_COEF2 + 2 * j);
          const float q = q2f<QT>(st.q<QT>(qb + j)[r]);
          qn = __fmaf_rn(c.x, q, qn);
          ql = __fmaf_rn(c.y, q, ql);
        }
        qn += ql;
        const QT qs = f2q<QT>(qn);
        outq<QT>(a, kk)[row] = qs;
        st.q<QT>(qb + kk)[r] = qs;
      }
      // v = w - Q coef (the coefficients are stored negated), added to w in FP64
      const double v = st.d(0)[r] + lp_chain<QT>(st, cf + CF_COEF + 2 * a.j0, qb, a.k - a.j0, r);
      {
        // the stored column v / ||Delta f||: (hi, lo) split of v times the
        // (hi, lo) scale on the FP32 pipe
        float p, e;
        prod_ff(d2f2(v), F2{cf[CF_MISC + 2], cf[CF_MISC + 3]}, p, e);
        outq<QT>(a, a.k)[row] = f2q<QT>(__fadd_rn(p, e));
      }
      dv0 = v;
      if (a.step_mode) {
        const double f = st.d(1)[r];
        dv1 = f;
        if (split & 2u) st.put(1, r, d2f2(f));  // f meets q_{k-1} (DCGS-2)
      }
      break;
    }
    case K_CGS2B: {
      const double y = st.d(0)[r] + lp_chain<QT>(st, cf + CF_COEF, a.qbase, a.k, r);
      a.out_df[row] = y;
      dv0 = y;
      if (split & 1u) st.put(0, r, d2f2(y));
      break;
    }
    case K_MGS: {
      const double v = st.d(0)[r] + lp_chain<QT>(st, cf + CF_COEF + 2 * (a.jm - 1), a.qbase, 1, r);
      a.out_df[row] = v;
      dv0 = v;
      if (split & 1u) st.put(0, r, d2f2(v));
      break;
    }
    case K_UPDATE: {
      const double xn = st.d(0)[r] + lp_chain<QT>(st, cf + CF_COEF, a.qbase, a.ng, r);
      a.out_x[row] = xn;
      if (a.stop_kind == 1) dv1 = xn - st.d(1)[r];
      break;
    }
    case K_LSQ: {
      dv0 = st.d(0)[r];
      if (split & 1u) st.put(0, r, d2f2(dv0));
      break;
    }
    default:
      break;
  }
}

// Row program of the first pass (K_A) for FP64 history with the rotation and
// the dot-product operands in (hi, lo) float arithmetic on the FP32/INT pipes
// (AA_FLAG_DF_ARITH; the other passes stay on row_program).  Stored doubles
// are split into float pairs (integer operations, 2^-48 relative), rotated
// with the multiply-adds of aa_df.cuh and joined back into doubles with one
// FP64 add; the residual differences f = g - x, df, dg stay exact FP64 adds.
// Returns the stage columns it left in shared memory as (hi, lo) pairs
// (bit c of cv[c >> 6]); the kernel splits the remaining dot columns itself.
__device__ __forceinline__ F2 cfpair(const float *cf, int i) { return F2{cf[i], cf[i + 1]}; }

__device__ __forceinline__ void row_program_dd(const PassArgs &a, Stage st, int t, int r,
                                               const double *co, const float *cf, uint64_t cv[2]) {
  const int64_t row = (int64_t)t * TR + r;
  auto mark = [&](int c) { cv[c >> 6] |= 1ull << (c & 63); };
  cv[0] = cv[1] = 0ull;
  if (a.kind != K_A) return;
  double df;
  if (a.step_mode) {
    const double x = st.d(0)[r], g = st.d(1)[r], gp = st.d(2)[r], fp = st.d(3)[r];
    const double f = g - x;
    df = f - fp;
    const double dg = g - gp;
    ((double *)a.out_dg)[row] = dg;
    a.out_f[row] = f;
    a.out_g[row] = g;
    st.put(0, r, d2f2(f));
    st.put(1, r, d2f2(df));
    mark(0);
    mark(1);
  } else {
    df = st.d(0)[r];
    st.put(0, r, d2f2(df));
    mark(0);
  }
  a.out_df[row] = df;
  if (a.k == 0) outq<double>(a, 0)[row] = df;
  if (a.del) {
    // the scaled Givens rotations of row_program, as (hi, lo) multiply-adds
    const int qb = a.qbase;
    F2 w = d2f2(st.d(qb)[r]);
    for (int j = 0; j < a.m - 1; ++j) {
      const F2 u = d2f2(st.d(qb + j + 1)[r]);
      const F2 k1 = cfpair(cf, CF_ROT + 4 * j), k2 = cfpair(cf, CF_ROT + 4 * j + 2);
      // both forms as one (operands selected, see row_program)
      const bool ty = __double_as_longlong(co[CO_ROT + 4 * j + 2]) != 0;
      const F2 P = df_mad(ty ? k1 : k2, u, w);   // w + kp u
      const F2 Qv = df_mad(ty ? k2 : k1, w, u);  // u + kq w
      const F2 out = ty ? P : Qv;
      w = ty ? Qv : P;
      outq<double>(a, j)[row] = f22d(out);
      st.put(qb + j, r, out);
      mark(qb + j);
    }
  }
}

// ------------------------------------------------------- m x m epilogues
//
// The small dense part of each add runs in the last CTA of a pass, by warp
// 0, on shared-memory copies of the m x m state (the stage buffers are free
// once the tile loop has ended).  Layout of the scratch (doubles, ld = M):
//   Rs[M*M], Ts[M*M], then vectors sig, rhs, rcol, gam, coef, s (M each).

__device__ __forceinline__ double &RR(double *A, int j, int l) { return A[j * MMAX + l]; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Epi {
  int M;
  double *R, *T, *sig, *rhs, *rcol, *gam, *coef, *s;
  __device__ double &r(int j, int l) const { return R[j * M + l]; }
  __device__ double &t(int j, int l) const { return T[j * M + l]; }
};

__host__ __device__ inline size_t epi_doubles(int M) { return (size_t)2 * M * M + 6 * (size_t)M + 8; }

static __device__ Epi epi_layout(double *base, int M) {
  Epi e;
  e.M = M;
  e.R = base;
  e.T = e.R + M * M;
  e.sig = e.T + M * M;
  e.rhs = e.sig + M;
  e.rcol = e.rhs + M;
  e.gam = e.rcol + M;
  e.coef = e.gam + M;
  e.s = e.coef + M;
  return e;
}

// Copy a ld-MMAX global matrix into a ld-M shared one (and back).
static __device__ void mat_in(double *dst, const double *src, int M, int lane) {
  for (int i = lane; i < M * M; i += 32) dst[i] = src[(i / M) * MMAX + (i % M)];
  __syncwarp();
}
// (Entries outside the leading M x M block are never written after the
// state is zeroed at creation and reset, and never read.)
static __device__ void mat_out(double *dst, const double *src, int M, int lane) {
  for (int i = lane; i < M * M; i += 32) dst[(i / M) * MMAX + (i % M)] = src[i];
  __syncwarp();
}
static __device__ void vec_in(double *dst, const double *src, int n, int lane) {
  for (int i = lane; i < n; i += 32) dst[i] = src[i];
  __syncwarp();
}
static __device__ void vec_out(double *dst, const double *src, int n, int lane) {
  for (int i = lane; i < n; i += 32) dst[i] = src[i];
  __syncwarp();
}

// The small triangular solves run by columns on warp 0: lane j keeps the
// partial right-hand side of rows j and j + 32 (n <= 64) in registers, so a
// step is one broadcast and one multiply-add instead of a warp reduction per
// row (on GB300 a dependent FP64 operation costs many cycles, and the m x m
// work sits on every pass's critical path).

// Back substitution with an upper-triangular R (ld M): x = R^{-1} b, n unknowns.
// The reciprocals of the diagonal are formed once, in parallel.
static __device__ void backsolve(const Epi &e, const double *b, double *x, int n, int lane) {
  double s0 = (lane < n) ? b[lane] : 0.0, s1 = (lane + 32 < n) ? b[lane + 32] : 0.0;
  const double i0 = (lane < n) ? 1.0 / e.R[lane * e.M + lane] : 0.0;
  const double i1 = (lane + 32 < n) ? 1.0 / e.R[(lane + 32) * e.M + lane + 32] : 0.0;
  for (int l = n - 1; l >= 0; --l) {
    const double own = (l >= 32) ? s1 * i1 : s0 * i0;  // x_l, valid on lane l % 32
    const double xl = __shfl_sync(0xffffffffu, own, l & 31);
    if (lane == (l & 31)) x[l] = xl;
    if (lane < l) s0 -= e.R[lane * e.M + l] * xl;
    if (lane + 32 < l) s1 -= e.R[(lane + 32) * e.M + l] * xl;
  }
  __syncwarp();
}

// Forward substitution with the unit-lower T (ld M): x = T^{-1} x in place.
static __device__ void forward_unit(const Epi &e, double *x, int n, int lane) {
  double v0 = (lane < n) ? x[lane] : 0.0, v1 = (lane + 32 < n) ? x[lane + 32] : 0.0;
  for (int l = 0; l + 1 < n; ++l) {
    const double xl = __shfl_sync(0xffffffffu, (l >= 32) ? v1 : v0, l & 31);
    if (lane > l && lane < n) v0 -= e.T[lane * e.M + l] * xl;
    if (lane + 32 > l && lane + 32 < n) v1 -= e.T[(lane + 32) * e.M + l] * xl;
  }
  __syncwarp();
  if (lane < n) x[lane] = v0;
  if (lane + 32 < n) x[lane + 32] = v1;
  __syncwarp();
}

// Givens parameters of the next QRDelete, computed from R alone: the rotated
// R, the per-row rotation coefficients folded with the stored columns'
// scales, and (ICWY) the correction matrix rotated at the m x m level.
// Runs when the history has just become full; overwrites e.R and e.T.
static __device__ void prepare_delete(const PassArgs &a, DevState *S, const Epi &e, int lane) {
  const int M = e.M;
  const bool icwy_rot = (a.orth == O_ICWY) && !(a.flags & 0x2u);
  // H = R without its first column (M x (M-1), upper Hessenberg), in place.
  for (int j = 0; j < M; ++j) {
    double v[2];
    int cnt = 0;
    for (int l = lane; l < M; l += 32) v[cnt++] = (l + 1 < M) ? e.r(j, l + 1) : 0.0;
    __syncwarp();
    cnt = 0;
    for (int l = lane; l < M; l += 32) e.r(j, l) = v[cnt++];
    __syncwarp();
  }
  if (icwy_rot) {
    // Gram of the stored columns 0..M-2 from T = I + L (strictly-lower part
    // kept in place, mirrored into the upper part); the delayed row of
    // column M-1 is still unknown and is left as an identity row/column.
    for (int i = lane; i < M * M; i += 32) {
      const int j = i / M, l = i % M;
      if (j < l) e.T[i] = (l < M - 1) ? e.t(l, j) : 0.0;
    }
    __syncwarp();
    for (int i = lane; i < M * M; i += 32) {
      const int j = i / M, l = i % M;
      if (j == l) e.T[i] = 1.0;
      else if (j > l && j == M - 1) e.T[i] = 0.0;
    }
    __syncwarp();
  }
  double tau = e.sig[0];  // scale of the carried column (lane 0 only)
  for (int j = 0; j + 1 < M; ++j) {
    const double av = e.r(j, j), bv = e.r(j + 1, j);
    // c = a / hypot(a, b), s = b / hypot(a, b) with one reciprocal square
    // root (a short dependency chain); hypot and divisions only where
    // a^2 + b^2 would leave the normal range
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
    for (int l = j + lane; l + 1 < M; l += 32) {
      const double hj = e.r(j, l), hj1 = e.r(j + 1, l);
      e.r(j, l) = c * hj + s * hj1;
      e.r(j + 1, l) = -s * hj + c * hj1;
    }
    __syncwarp();
    if (lane == 0) {
      e.r(j + 1, j) = 0.0;
      // scaled rotation of (carry, column j+1): carry has scale tau, the
      // stored column j+1 has scale sig_{j+1}; pick the form whose
      // multipliers stay bounded.
      const double sj1 = e.sig[j + 1];
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
      S->rot[4 * j + 0] = k1;
      S->rot[4 * j + 1] = k2;
      S->rot[4 * j + 2] = type;
      S->rot[4 * j + 3] = sout;
    }
    if (icwy_rot) {
      for (int i = lane; i < M; i += 32) {  // columns j, j+1
        const double gj = e.t(i, j), gj1 = e.t(i, j + 1);
        e.t(i, j) = c * gj + s * gj1;
        e.t(i, j + 1) = -s * gj + c * gj1;
      }
      __syncwarp();
      for (int l = lane; l < M; l += 32) {  // rows j, j+1
        const double gj = e.t(j, l), gj1 = e.t(j + 1, l);
        e.t(j, l) = c * gj + s * gj1;
        e.t(j + 1, l) = -s * gj + c * gj1;
      }
    }
    __syncwarp();
  }
  for (int l = lane; l < M; l += 32) e.r(M - 1, l) = 0.0;
  __syncwarp();
  mat_out(S->Rn, e.R, M, lane);
  if (icwy_rot) {
    // T' = I + strictly-lower Gram of the rotated columns 0..M-3; row M-2 is
    // the delayed row that the next add computes.
    for (int i = lane; i < M * M; i += 32) {
      const int j = i / M, l = i % M;
      double v = 0.0;
      if (j == l && j < M - 1) v = 1.0;
      else if (l < j && j <= M - 3) v = e.T[i];
      e.T[i] = v;
    }
    __syncwarp();
    mat_out(S->Tn, e.T, M, lane);
  }
  if (lane == 0) {
    S->rot0 = e.sig[0];
    S->pend_del = 1;
  }
  __syncwarp();
}

// Finish a QRAdd: diagonal entry, breakdown test, the least-squares solve of
// Algorithm 2 (step mode) and gamma in dG slot order.  e holds R, T, sig,
// rhs and rcol for the current add.
static __device__ void finalize_add(const PassArgs &a, DevState *S, const Epi &e, double rho, double vf,
                             double vscale, double qnf, int lane) {
  const int k = a.k, m = a.m;
  const double dfn = sqrt(S->st.dfnorm2);
  const bool bd = !(rho > 0.0) || !isfinite(rho) || rho <= a.breakdown_tol * dfn;
  if (bd) {
    for (int j = lane; j < MMAX; j += 32) S->gphys[j] = 0.0;
    if (lane == 0) {
      S->st.rho = rho;
      S->st.breakdown = 1;
      S->st.cols = 0;
      S->pend_del = 0;
    }
    __syncwarp();
    return;
  }
  for (int l = lane; l < m; l += 32) e.r(k, l) = 0.0;
  __syncwarp();
  for (int j = lane; j < k; j += 32) e.r(j, k) = e.rcol[j];
  if (lane == 0) {
    e.r(k, k) = rho;
    e.sig[k] = 1.0 / (rho * vscale);
  }
  if (a.orth == O_ICWY) {
    for (int l = lane; l < m; l += 32) e.t(k, l) = (l == k) ? 1.0 : 0.0;
  }
  __syncwarp();
  if (a.step_mode) {
    if (lane == 0) {
      e.rhs[k] = vf / rho;
      if (a.orth == O_DCGS2 && (a.flags & 0x100u)) e.rhs[k - 1] = qnf;
    }
    __syncwarp();
    backsolve(e, e.rhs, e.gam, k + 1, lane);
    for (int j = lane; j < MMAX; j += 32) S->gphys[j] = 0.0;
    __syncwarp();
    for (int j = lane; j <= k; j += 32) S->gphys[(a.head_new + j) % m] = e.gam[j];
    vec_out(S->rhs, e.rhs, k + 1, lane);
    vec_out(S->gam, e.gam, k + 1, lane);
  }
  mat_out(S->R, e.R, m, lane);
  if (a.orth == O_ICWY) mat_out(S->T, e.T, m, lane);
  vec_out(S->sig, e.sig, k + 1, lane);
  if (lane == 0) {
    S->st.rho = rho;
    S->st.breakdown = 0;
    S->st.cols = k + 1;
  }
  __syncwarp();
  if (k + 1 == m) prepare_delete(a, S, e, lane);
}

// Warp 0 of the last CTA.
static __device__ void epilogue(const PassArgs &a, double *scratch, int lane) {
  DevState *S = a.st;
  const double *red = S->red;
  const int k = a.k;
  const int m = a.m;
  Epi e = epi_layout(scratch, m > 0 ? m : 1);
  switch (a.kind) {
    case K_INIT: {
      if (lane == 0) {
        S->st.fnorm2 = red[0];
        if (!isfinite(red[0])) S->st.status = DEV_ENONFINITE;
      }
      break;
    }
    case K_A: {
      const int o = a.step_mode ? 1 : 0;
      const double dfn2 = red[o];
      const double fn2 = a.step_mode ? red[0] : 0.0;
      if (lane == 0) {
        if (a.step_mode) S->st.fnorm2 = fn2;
        S->st.dfnorm2 = dfn2;
      }
      if (!isfinite(dfn2) || !isfinite(fn2)) {
        for (int j = lane; j < MMAX; j += 32) S->gphys[j] = 0.0;
        if (lane == 0) {
          S->st.status = DEV_ENONFINITE;
          S->st.breakdown = 1;
          S->st.cols = 0;
          S->pend_del = 0;
        }
        break;
      }
      // current state -> shared memory (after a delete: the pending rotated R/T)
      mat_in(e.R, a.del ? S->Rn : S->R, m, lane);
      if (a.orth == O_ICWY) mat_in(e.T, (a.del && !(a.flags & 0x2u)) ? S->Tn : S->T, m, lane);
      vec_in(e.sig, S->sig, m, lane);
      vec_in(e.rcol, S->rcol, m, lane);
      if (a.del) {
        for (int j = lane; j < k; j += 32) e.sig[j] = S->rot[4 * j + 3];
        if (lane == 0) S->pend_del = 0;
        __syncwarp();
      }
      if (k == 0) {
        finalize_add(a, S, e, sqrt(dfn2), a.step_mode ? red[2] : 0.0, 1.0, 0.0, lane);
        break;
      }
      if (a.step_mode)
        for (int j = lane; j < k; j += 32) e.rhs[j] = e.sig[j] * red[a.off_rhs + j];
      if (lane == 0) S->vscale = dfn2 > 0.0 ? 1.0 / sqrt(dfn2) : 1.0;
      __syncwarp();
      switch (a.orth) {
        case O_MGS: {
          if (lane == 0) {
            const double r0 = e.sig[0] * red[a.off_r];
            S->rcol[0] = r0;
            S->coef[0] = r0 * e.sig[0];
          }
          break;
        }
        case O_ICWY: {
          if ((a.flags & 0x2u) && a.del) {
            // T refreshed from the Gram reduction of the rotated factor
            for (int i = lane; i < m * m; i += 32) e.T[i] = ((i / m) == (i % m)) ? 1.0 : 0.0;
            __syncwarp();
            if (lane == 0) {
              int g = 0;
              for (int j = 1; j <= k - 2; ++j)
                for (int l = 0; l < j; ++l) e.t(j, l) = red[a.off_gram + g++];
            }
            __syncwarp();
          }
          for (int l = lane; l < m; l += 32)
            e.t(k - 1, l) = (l + 1 < k) ? e.sig[l] * e.sig[k - 1] * red[a.off_t + l]
                                        : ((l == k - 1) ? 1.0 : 0.0);
          for (int j = lane; j < k; j += 32) e.rcol[j] = e.sig[j] * red[a.off_r + j];
          __syncwarp();
          forward_unit(e, e.rcol, k, lane);
          for (int j = lane; j < k; j += 32) e.coef[j] = e.sig[j] * e.rcol[j];
          __syncwarp();
          mat_out(S->T, e.T, m, lane);
          vec_out(S->rcol, e.rcol, k, lane);
          vec_out(S->coef, e.coef, k, lane);
          break;
        }
        case O_CGS2: {
          for (int j = lane; j < k; j += 32) {
            const double sj = e.sig[j] * red[a.off_r + j];
            S->s[j] = sj;
            S->coef[j] = e.sig[j] * sj;
          }
          break;
        }
        default: {  // DCGS-2
          for (int j = lane; j < k; j += 32) e.rcol[j] = e.sig[j] * red[a.off_r + j];
          const bool reorth = (a.flags & 0x100u) != 0;
          __syncwarp();
          if (reorth) {
            const double rkk = e.r(k - 1, k - 1);
            const double sk = e.sig[k - 1];
            for (int j = lane; j < k - 1; j += 32) {
              const double sj = e.sig[j] * sk * red[a.off_s + j];
              S->s[j] = sj;
              e.r(j, k - 1) += (a.flags & 0x1u) ? rkk * sj : sj;
              S->coef2[j] = sj * e.sig[j];
            }
            __syncwarp();
            if (lane == 0) {
              S->rcself = sk;
              e.sig[k - 1] = 1.0;
            }
            __syncwarp();
          }
          for (int j = lane; j < k; j += 32) e.coef[j] = e.rcol[j] * e.sig[j];
          __syncwarp();
          vec_out(S->rcol, e.rcol, k, lane);
          vec_out(S->coef, e.coef, k, lane);
          if (lane == 0) S->reorth = reorth;
          break;
        }
      }
      __syncwarp();
      mat_out(S->R, e.R, m, lane);
      vec_out(S->sig, e.sig, m, lane);
      if (a.step_mode) vec_out(S->rhs, e.rhs, k, lane);
      break;
    }
    case K_CGS2B: {
      for (int j = lane; j < k; j += 32) {
        const double z = S->sig[j] * red[j];
        S->rcol[j] = S->s[j] + z;
        S->coef[j] = S->sig[j] * z;
      }
      break;
    }
    case K_MGS: {
      if (lane == 0) {
        const double r = S->sig[a.jm] * red[0];
        S->rcol[a.jm] = r;
        S->coef[a.jm] = r * S->sig[a.jm];
      }
      break;
    }
    case K_PROJ: {
      const double vn2 = red[0];
      const double vf = a.step_mode ? red[1] : 0.0;
      const double qnf = (a.step_mode && a.orth == O_DCGS2 && (a.flags & 0x100u)) ? red[2] : 0.0;
      mat_in(e.R, S->R, m, lane);
      if (a.orth == O_ICWY) mat_in(e.T, S->T, m, lane);
      vec_in(e.sig, S->sig, m, lane);
      vec_in(e.rcol, S->rcol, m, lane);
      vec_in(e.rhs, S->rhs, m, lane);
      finalize_add(a, S, e, sqrt(vn2), vf, S->vscale, qnf, lane);
      break;
    }
    case K_UPDATE: {
      if (lane == 0) S->st.xdiff2 = red[0];
      break;
    }
    case K_LSQ: {
      const int c = a.c;
      mat_in(e.R, S->R, m, lane);
      for (int j = lane; j < c; j += 32) e.rhs[j] = S->sig[j] * red[j];
      __syncwarp();
      backsolve(e, e.rhs, e.gam, c, lane);
      vec_out(S->rhs, e.rhs, c, lane);
      vec_out(S->gam, e.gam, c, lane);
      break;
    }
    case K_MDOT: {
      for (int d = lane; d < a.ndots; d += 32) a.result_host_dev[d] = red[d];
      break;
    }
    default:
      break;
  }
  __syncwarp();
}

// Passes of the exact-FP64 form with at most RD dot products (projection,
// update, MGS links, the first add) accumulate them in the row program's own
// thread, row by row, instead of in a separate warp-per-dot phase: no second
// barrier per tile and no warps idling while one or two warps sum the tile.
// (The float-pair forms keep the dot phase: there the per-row compensated
// sums measured slower.)
constexpr int RD = 4;

// MODE 1 operand scaling.  The FP32-pipe products need operands well inside
// the float range, so every split column is scaled by a power of two 2^s
// (exact; the sums are scaled back by 2^-(s_a + s_b)).  Stored history
// columns u_j (q_j = sig_j u_j, so ||u_j|| = 1 / sig_j) are brought to a
// root-mean-square entry near 1.  The vectors f, Delta f (pass A) and y
// (CGS-2 middle pass) are brought near 2^16 from the squared norm of the
// previous pass A (f and Delta f of consecutive iterations have similar
// sizes) or the current ||Delta f||^2: since |a 2^s| in [2^-74, 2^128) is
// split exactly, a vector may be up to about 2^90 smaller or 2^47 larger
// (cross products below 2^127) than that estimate.
__device__ __forceinline__ int pow2_of_rms(double mean_sq, bool inverse, int centre) {
  if (!(mean_sq > 0.0) || !(mean_sq < 1e300)) return centre;
  const int ex = ((__double2hiint(mean_sq) >> 20) & 0x7ff) - 1023;  // floor(log2 mean_sq)
  const int s = (inverse ? (ex >> 1) : -(ex >> 1)) + centre;
  return max(-400, min(400, s));
}

static __device__ int dot_col_exp(const PassArgs &a, const DevState *S, int c) {
  const double n = (double)a.n;
  if (c < a.qbase) {
    const double v2 = (a.kind == K_A && a.step_mode) ? S->st.fnorm2 : S->st.dfnorm2;
    return pow2_of_rms(v2 / n, false, 16);
  }
  const int j = c - a.qbase;
  if (j >= MMAX) return 0;
  const double sg = (a.kind == K_A && a.del) ? (j < a.m - 1 ? S->rot[4 * j + 3] : 0.0) : S->sig[j];
  // mean square of u_j = 1 / (sig_j^2 n): scale by sqrt(sig_j^2 n)
  return pow2_of_rms(sg * sg * n, true, 0);
}

// A float partial sum into FP64 (exact), by integer operations: the
// hardware conversion runs on the FP64 pipe, which is the scarce unit here.
template <int MODE>
__device__ __forceinline__ double fold_f(float x) {
  return f2d(x);
}

// 2^e as a double, e in [-1022, 1023] (exact).
__device__ __forceinline__ double pow2d(int e) {
  return __hiloint2double((1023 + e) << 20, 0);
}

// One dot product of the FP32-pipe dot phase (MODES 1-3) over one tile:
// (S2, C2) += sum over the tile's rows of column ca times column cb, the
// columns read from the stage as stored history (FP32/BF16, MODE 2) or as
// (hi, lo) splits of FP64 columns.
template <class QT, int MODE>
__device__ __forceinline__ void dot_tile(Stage st, int ca, int cb, int qbase, int rows, int lane,
                                         float2 &S2, float2 &C2) {
  const bool qa = (MODE == 2) && ca >= qbase, qb = (MODE == 2) && cb >= qbase;
  if (rows == TR) {
    // full tile: lane l takes row pairs 2l + 64h (8-byte history
    // loads, 16-byte split-pair loads, contiguous across the warp)
    // and works on both rows with paired FP32 instructions
    float2 p, e;
    // MODE 2: the row pairs at even and odd h go to two compensated chains
    // (the second one merged at the end) so that two independent dependency
    // chains run per dot
    float2 Sb = make_float2(0.f, 0.f), Cb = make_float2(0.f, 0.f);
    if (qa && qb) {
#pragma unroll
      for (int h = 0; h < TR / 64; h += 2) {
        const int r = 2 * lane + 64 * h;
        const float2 x = q2rows<QT>(st, ca, r), y = q2rows<QT>(st, cb, r);
        const float2 x1 = q2rows<QT>(st, ca, r + 64), y1 = q2rows<QT>(st, cb, r + 64);
        p = __fmul2_rn(x, y);
        const float2 p1 = __fmul2_rn(x1, y1);
        e = __ffma2_rn(x, y, neg2(p));
        const float2 e1 = __ffma2_rn(x1, y1, neg2(p1));
        acc_add2(S2, C2, p, e);
        acc_add2(Sb, Cb, p1, e1);
      }
      acc_add2(S2, C2, Sb, Cb);
    } else if (qa || qb) {
      const int cq = qa ? ca : cb, cv = qa ? cb : ca;
#pragma unroll
      for (int h = 0; h < TR / 64; h += 2) {
        const int r = 2 * lane + 64 * h;
        const float2 q = q2rows<QT>(st, cq, r), q1 = q2rows<QT>(st, cq, r + 64);
        const float4 v = st.pairs2(cv, r), v1 = st.pairs2(cv, r + 64);
        float2 p1, e1;
        prod_f2(make_float2(v.x, v.y), make_float2(v.z, v.w), q, p, e);
        prod_f2(make_float2(v1.x, v1.y), make_float2(v1.z, v1.w), q1, p1, e1);
        acc_add2(S2, C2, p, e);
        acc_add2(Sb, Cb, p1, e1);
      }
      acc_add2(S2, C2, Sb, Cb);
    } else if constexpr (MODE == 1) {
      // FP64 storage: one compensated pair per dot (registers for
      // four CTAs per SM, which the FP64 rotation chains need more
      // than the paired instructions)
      float S = S2.x, C = C2.x, ps, es;
#pragma unroll
      for (int h = 0; h < TR / 64; ++h) {
        const int r = 2 * lane + 64 * h;
        const float4 x = st.pairs2(ca, r), y = st.pairs2(cb, r);
        prod_ff(F2{x.x, x.z}, F2{y.x, y.z}, ps, es);
        acc_add(S, C, ps, es);
        prod_ff(F2{x.y, x.w}, F2{y.y, y.w}, ps, es);
        acc_add(S, C, ps, es);
      }
      S2.x = S;
      C2.x = C;
    } else {
#pragma unroll
      for (int h = 0; h < TR / 64; ++h) {
        const int r = 2 * lane + 64 * h;
        const float4 x = st.pairs2(ca, r), y = st.pairs2(cb, r);
        prod_ff2(make_float2(x.x, x.y), make_float2(x.z, x.w), make_float2(y.x, y.y),
                 make_float2(y.z, y.w), p, e);
        acc_add2(S2, C2, p, e);
      }
    }
  } else {
    // ragged last tile: one row at a time, into the even-row sums
    float S = S2.x, C = C2.x, p, e;
    if (qa && qb) {
      for (int r = lane; r < rows; r += 32) {
        const float x = q2f<QT>(st.q<QT>(ca)[r]), y = q2f<QT>(st.q<QT>(cb)[r]);
        p = __fmul_rn(x, y);
        e = __fmaf_rn(x, y, -p);
        acc_add(S, C, p, e);
      }
    } else if (qa || qb) {
      const int cq = qa ? ca : cb, cv = qa ? cb : ca;
      for (int r = lane; r < rows; r += 32) {
        prod_f(st.f2(cv, r), q2f<QT>(st.q<QT>(cq)[r]), p, e);
        acc_add(S, C, p, e);
      }
    } else {
      for (int r = lane; r < rows; r += 32) {
        prod_ff(st.f2(ca, r), st.f2(cb, r), p, e);
        acc_add(S, C, p, e);
      }
    }
    S2.x = S;
    C2.x = C;
  }
}

// Dot-product families of the FP32/BF16-history form (MODE 2).  A pass's
// phase dots are q_j . v for history columns q_j (stage column qbase + j) and
// at most three shared vectors v: NS split FP64 vectors (f, Delta f, or the
// projected vector; (hi, lo) pairs in the stage) and, with HQ, one history
// column (q_{k-1}: ICWY's T row, DCGS-2's correction coefficients).  Warp w
// takes the columns j = w, w + NWARP, w + 2 NWARP (ncw of them) and every
// vector, so the vectors are loaded once per row pair for all of the warp's
// columns, each column once for all vectors, and up to nine independent
// compensated chains run side by side.  A (column, vector) pair without a
// dot product is computed and dropped.  Accumulator slot 3c + vi belongs to
// the warp's column c and vector vi (vi = 0, 1 split, 2 history).
constexpr int FAM_COLS = 3;                 // columns per warp
constexpr int FAM_SLOTS = 3 * FAM_COLS;     // accumulator slots per lane
constexpr int FAM_MAXJ = NWARP * FAM_COLS;  // history columns a family may span

template <class QT, int NS, bool HQ>
__device__ __forceinline__ void fam_tile(Stage st, const int (&col)[FAM_COLS], int ncw, int v0,
                                         int v1, int vq, int rows, int lane,
                                         float2 (&S)[FAM_SLOTS], float2 (&C)[FAM_SLOTS]) {
  if (rows == TR) {
#pragma unroll
    for (int h = 0; h < TR / 64; ++h) {
      const int r = 2 * lane + 64 * h;
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      float2 aq = make_float2(0.f, 0.f);
      if (NS >= 1) a0 = st.pairs2(v0, r);
      if (NS >= 2) a1 = st.pairs2(v1, r);
      if (HQ) aq = q2rows<QT>(st, vq, r);
#pragma unroll
      for (int c = 0; c < FAM_COLS; ++c) {
        if (c < ncw) {
          const float2 x = q2rows<QT>(st, col[c], r);
          float2 p, e;
          if (NS >= 1) {
            prod_f2(make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), x, p, e);
            acc_add2(S[3 * c], C[3 * c], p, e);
          }
          if (NS >= 2) {
            prod_f2(make_float2(a1.x, a1.y), make_float2(a1.z, a1.w), x, p, e);
            acc_add2(S[3 * c + 1], C[3 * c + 1], p, e);
          }
          if (HQ) {
            p = __fmul2_rn(x, aq);
            e = __ffma2_rn(x, aq, neg2(p));
            acc_add2(S[3 * c + 2], C[3 * c + 2], p, e);
          }
        }
      }
    }
  } else {
    // ragged last tile: one row at a time, into the even-row sums
    for (int r = lane; r < rows; r += 32) {
      F2 b0{0.f, 0.f}, b1{0.f, 0.f};
      float bq = 0.f;
      if (NS >= 1) b0 = st.f2(v0, r);
      if (NS >= 2) b1 = st.f2(v1, r);
      if (HQ) bq = q2f<QT>(st.q<QT>(vq)[r]);
#pragma unroll
      for (int c = 0; c < FAM_COLS; ++c) {
        if (c < ncw) {
          const float x = q2f<QT>(st.q<QT>(col[c])[r]);
          float p, e;
          if (NS >= 1) {
            prod_f(b0, x, p, e);
            acc_add(S[3 * c].x, C[3 * c].x, p, e);
          }
          if (NS >= 2) {
            prod_f(b1, x, p, e);
            acc_add(S[3 * c + 1].x, C[3 * c + 1].x, p, e);
          }
          if (HQ) {
            p = __fmul_rn(x, bq);
            e = __fmaf_rn(x, bq, -p);
            acc_add(S[3 * c + 2].x, C[3 * c + 2].x, p, e);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- kernel
//
// MODE 0: FP64 storage, FP64 arithmetic throughout (exact FP64 path).
// MODE 1: FP64 storage and FP64 row programs (rotation, differences, all
//         stored values exact FP64), for passes with more than RD dot
//         products (AA_FLAG_FP32_DOTS): the leading squared norms of vectors
//         stay FP64 row-local sums (they also carry the non-finite test);
//         the other dot products run on the FP32 pipe from scaled (hi, lo)
//         splits (d2f2_dot), exact head products, compensated per-lane
//         float-pair sums folded into FP64 every eighth tile.
// MODE 2: FP32/BF16 storage; row programs and dot products on the FP32/INT
//         pipes (row_program_df), partial sums folded into FP64 every
//         second tile.
// MODE 3: FP64 storage, first pass only (AA_FLAG_DF_ARITH): rotation and dot
//         products on the FP32/INT pipes (row_program_dd), partial sums
//         folded into FP64 every fourth tile.

// Register budgets: the FP32-pipe forms (MODE 2, 3) hold two compensated float
// pairs per dot product (one per row parity), so their 4- and 8-dot buckets
// are held to 80 registers (3 CTAs per SM, no spills) and the 16-dot bucket to
// one CTA; MODE 1's 8-dot bucket (one pair per dot) to 64 (4 CTAs);
// every other instantiation keeps the compiler's own choice (a minimum of 0
// blocks states no bound: an explicit 1 lets it grow the FP64 projection and
// update from 48 to 80 registers and cost them a resident CTA).
template <class QT, int DPW, int MODE = 0>
__global__ void __launch_bounds__(NT, (MODE != 0)
                                          ? ((MODE == 1 && DPW == 8) ? 4 : (DPW > 1 && DPW <= 8) ? 3 : (DPW == 16 ? 1 : 0))
                                          : 0)
    pass_kernel(const __grid_constant__ PassArgs a, int nstages) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[STAGES];
  __shared__ double co[CO_SIZE];
  __shared__ __align__(16) float cf[MODE >= 2 ? CF_SIZE : 4];
  __shared__ uint8_t sda[NDOT_MAX], sdb[NDOT_MAX];
  __shared__ int s_last;
  __shared__ int s_err;
  // MODE 1: per-column split constants and scale exponents, the columns to
  // split, and the number of leading FP64 squared-norm dots
  __shared__ uint32_t s_sb[MODE == 1 ? MAXCOL : 1], s_lim[MODE == 1 ? MAXCOL : 1];
  __shared__ int s_cexp[MODE == 1 ? MAXCOL : 1];
  __shared__ uint64_t s_split[2];
  __shared__ int s_n64;
  __shared__ uint64_t s_tymask;  // bit j: form of QRDelete rotation j (MODE 2)
  // MODE 2 dot-product family: s_fam = {on, split vectors, history vector,
  // vector columns x3}; s_famd[vi][j] = dot of column j with vector vi (-1: none)
  __shared__ int s_fam[MODE == 2 ? 6 : 1];
  __shared__ int16_t s_famd[MODE == 2 ? 3 : 1][MODE == 2 ? FAM_MAXJ : 1];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const size_t stage_bytes = stage_size<QT>(a);
  DevState *S = a.st;

  // Per-pass coefficients from the device state (written by earlier passes).
  for (int i = tid; i < CO_SIZE; i += NT) co[i] = 0.0;
  for (int d = tid; d < a.ndots; d += NT) {
    sda[d] = a.dot_a[d];
    sdb[d] = a.dot_b[d];
  }
  if (tid == 0) s_err = 0;
  if constexpr (MODE == 1) {
    for (int c = tid; c < a.ncol; c += NT) {
      const int e = dot_col_exp(a, S, c);
      s_cexp[c] = e;
      s_sb[c] = (uint32_t)(128 + e) << 23;
      s_lim[c] = (uint32_t)(949 - e) << 20;
    }
    if (tid == 0) {
      int n64 = 0;
      while (n64 < a.ndots && n64 < RD && a.dot_a[n64] == a.dot_b[n64] && a.dot_a[n64] < a.qbase)
        ++n64;
      uint64_t sm[2] = {0ull, 0ull};
      for (int d = n64; d < a.ndots; ++d) {
        sm[a.dot_a[d] >> 6] |= 1ull << (a.dot_a[d] & 63);
        sm[a.dot_b[d] >> 6] |= 1ull << (a.dot_b[d] & 63);
      }
      s_split[0] = sm[0];
      s_split[1] = sm[1];
      s_n64 = n64;
    }
  }
  if constexpr (MODE == 2) {
    // leading dots of two FP64 vectors: FP64 row-local sums; FP64 columns
    // that meet a history column in a later dot are split for the dot phase.
    // A pass with at most RD dots whose operands are all history columns or
    // FP64 columns 0 and 1 (an MGS link, a projection) takes every dot as an
    // FP64 row-local sum (history entries converted exactly), and so has no
    // dot phase and no barrier before it.
    if (tid == 0) {
      int n64 = 0;
      bool rowable = a.ndots <= RD;
      for (int d = 0; d < a.ndots && rowable; ++d)
        rowable = (a.dot_a[d] >= a.qbase || a.dot_a[d] < 2) && (a.dot_b[d] >= a.qbase || a.dot_b[d] < 2);
      if (rowable) n64 = a.ndots;
      while (n64 < a.ndots && n64 < RD && a.dot_a[n64] < a.qbase && a.dot_b[n64] < a.qbase &&
             a.dot_a[n64] < 2 && a.dot_b[n64] < 2)
        ++n64;
      uint64_t sm = 0ull;
      for (int d = n64; d < a.ndots; ++d) {
        if (a.dot_a[d] < a.qbase) sm |= 1ull << a.dot_a[d];
        if (a.dot_b[d] < a.qbase) sm |= 1ull << a.dot_b[d];
      }
      s_split[0] = sm;
      s_split[1] = 0ull;
      s_n64 = n64;
      // dot-product family (fam_tile): every phase dot is (history column,
      // shared vector) with at most two split vectors and one history vector,
      // no pair twice, and columns j < FAM_MAXJ
      int fam = (DPW == 4 || DPW == 8) ? 1 : 0;
      int vcol[3] = {-1, -1, -1};  // split vectors in slots 0, 1; history vector in slot 2
      int nsp = 0;
      for (int v = 0; v < 3; ++v)
        for (int j = 0; j < FAM_MAXJ; ++j) s_famd[v][j] = -1;
      for (int d = n64; d < a.ndots && fam; ++d) {
        const int ca = a.dot_a[d], cb = a.dot_b[d];
        const int j = ca - a.qbase;
        if (ca < a.qbase || j >= FAM_MAXJ) {
          fam = 0;
          break;
        }
        int vi = -1;
        if (cb >= a.qbase) {
          if (vcol[2] < 0) vcol[2] = cb;
          vi = (vcol[2] == cb) ? 2 : -1;
        } else {
          for (int v = 0; v < nsp; ++v)
            if (vcol[v] == cb) vi = v;
          if (vi < 0 && nsp < 2) {
            vcol[nsp] = cb;
            vi = nsp++;
          }
        }
        if (vi < 0 || s_famd[vi][j] >= 0) {
          fam = 0;
          break;
        }
        s_famd[vi][j] = (int16_t)d;
      }
      if (n64 >= a.ndots || nsp == 0) fam = 0;
      s_fam[0] = fam;
      s_fam[1] = nsp;
      s_fam[2] = vcol[2] >= 0 ? 1 : 0;
      s_fam[3] = vcol[0];
      s_fam[4] = vcol[1];
      s_fam[5] = vcol[2];
    }
  }
  __syncthreads();
  if (a.kind == K_A && a.del) {
    for (int i = tid; i < 4 * (a.m - 1); i += NT) co[CO_ROT + i] = S->rot[i];
    if (tid == 0) {
      co[CO_ROT0] = S->rot0;
      uint64_t tm = 0ull;
      for (int j = 0; j + 1 < a.m; ++j)
        if (__double_as_longlong(S->rot[4 * j + 2]) != 0) tm |= 1ull << j;
      s_tymask = tm;
    }
  } else if (a.kind == K_PROJ || a.kind == K_CGS2B || a.kind == K_MGS) {
    for (int i = tid; i < a.k; i += NT) {
      co[CO_COEF + i] = S->coef[i];
      co[CO_COEF2 + i] = S->coef2[i];
    }
    if (tid == 0) {
      co[CO_MISC] = S->rcself;
      co[CO_MISC + 1] = S->vscale;
    }
  } else if (a.kind == K_UPDATE) {
    for (int i = tid; i < a.ng; i += NT) co[CO_COEF + i] = S->gphys[a.pslot[i]];
  }
  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if constexpr (MODE >= 2) {
    // (hi, lo) float copies of the coefficients; projection/update
    // coefficients negated.
    for (int j = tid; j < MMAX; j += NT) {
      if (j < a.m - 1) {
        const F2 k1 = d2f2(co[CO_ROT + 4 * j]), k2 = d2f2(co[CO_ROT + 4 * j + 1]);
        cf[CF_ROT + 4 * j] = k1.h;
        cf[CF_ROT + 4 * j + 1] = k1.l;
        cf[CF_ROT + 4 * j + 2] = k2.h;
        cf[CF_ROT + 4 * j + 3] = k2.l;
      }
      const F2 c1 = d2f2(-co[CO_COEF + j]), c2 = d2f2(-co[CO_COEF2 + j]);
      cf[CF_COEF + 2 * j] = c1.h;
      cf[CF_COEF + 2 * j + 1] = c1.l;
      cf[CF_COEF2 + 2 * j] = c2.h;
      cf[CF_COEF2 + 2 * j + 1] = c2.l;
    }
    if (tid == 0) {
      const F2 rc = d2f2(co[CO_MISC]), vs = d2f2(co[CO_MISC + 1]);
      cf[CF_MISC] = rc.h;
      cf[CF_MISC + 1] = rc.l;
      cf[CF_MISC + 2] = vs.h;
      cf[CF_MISC + 3] = vs.l;
    }
    __syncthreads();
  }

  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < a.ntiles) issue_tile<QT>(a, Stage{smem + s * stage_bytes, a.qbase}, t, &bars[s]);
    }
  }

  // slots of per-lane dot-phase accumulators; the MODE 2 family form
  // (fam_tile) needs FAM_SLOTS of them
  constexpr int NSLOT = (MODE == 2 && (DPW == 4 || DPW == 8)) ? FAM_SLOTS : DPW;
  // FP64 sums of the dot phase: per lane in registers (MODES 0, 1, 3), or,
  // for MODE 2, summed over the warp at each fold into shared memory (frees
  // the registers for the family form's nine chains)
  constexpr bool SACC = (MODE == 2);
  double acc[SACC ? 1 : DPW];
  __shared__ double s_acc[SACC ? NWARP : 1][SACC ? NSLOT : 1];
  // FP32-pipe partial sums: (S, C) compensated pairs, one per row parity
  // (.x even rows, .y odd rows) so that full tiles use paired instructions
  float2 accS[MODE ? NSLOT : 1], accC[MODE ? NSLOT : 1];
  constexpr int NRD = ((DPW == 1 && MODE == 0) || MODE == 1 || MODE == 2) ? RD : 1;
  // every dot product accumulated row by row in FP64 (no dot phase)
  const bool rowdots = ((DPW == 1) && (MODE == 0) && a.ndots <= RD) ||
                       (MODE == 2 && s_n64 == a.ndots);
  // first dot of the warp-per-dot phase (MODE 1, 2: after the FP64 row dots)
  const int dbase = (MODE == 1 || MODE == 2) ? s_n64 : 0;
  double racc[NRD];
#pragma unroll
  for (int d = 0; d < NRD; ++d) racc[d] = 0.0;
#pragma unroll
  for (int i = 0; i < (SACC ? 1 : DPW); ++i) acc[i] = 0.0;
  if constexpr (SACC) {
    for (int i = lane; i < NSLOT; i += 32) s_acc[warp][i] = 0.0;
  }
  if constexpr (MODE != 0) {
#pragma unroll
    for (int i = 0; i < NSLOT; ++i) accS[i] = accC[i] = make_float2(0.f, 0.f);
  }
  constexpr int FLUSH = (MODE == 3) ? 4 : 8;  // tiles per fold into FP64
  // MODE 2 family form: this warp's columns (fam_tile)
  const bool famon = (MODE == 2) && !rowdots && s_fam[0] != 0;
  int fcol[FAM_COLS];
  int ncw = 0;
  if constexpr (MODE == 2) {
#pragma unroll
    for (int c = 0; c < FAM_COLS; ++c) {
      const int j = warp + NWARP * c;
      fcol[c] = a.qbase + j;
      if (famon && (s_famd[0][j] >= 0 || s_famd[1][j] >= 0 || s_famd[2][j] >= 0)) ncw = c + 1;
    }
  }
  // slot i of this warp's dot-phase accumulators holds dot slot_dot(i)
  // (a.ndots: none)
  auto slot_dot = [&](int i) -> int {
    if constexpr (MODE == 2) {
      if (famon) {
        const int d = s_famd[i % 3][warp + NWARP * (i / 3)];
        return d >= 0 ? d : a.ndots;
      }
    }
    return i < DPW ? min(dbase + warp + NWARP * i, (int)a.ndots) : (int)a.ndots;
  };
  // FP32-pipe forms: fold the per-lane float pairs into FP64 (exact
  // conversions); MODE 2 sums them over the warp (fixed butterfly) into
  // s_acc, the other forms keep per-lane sums
  auto fold_slots = [&](bool reset) {
    if constexpr (MODE != 0) {
#pragma unroll
      for (int i = 0; i < NSLOT; ++i) {
        if (slot_dot(i) < a.ndots) {
          if constexpr (SACC) {
            double v = (fold_f<MODE>(accS[i].x) + fold_f<MODE>(accS[i].y)) +
                       (fold_f<MODE>(accC[i].x) + fold_f<MODE>(accC[i].y));
            v = warp_sum(v);
            if (lane == 0) s_acc[warp][i] += v;
          } else {
            acc[i] += fold_f<MODE>(accS[i].x) + fold_f<MODE>(accS[i].y);
            acc[i] += fold_f<MODE>(accC[i].x) + fold_f<MODE>(accC[i].y);
          }
          if (reset) accS[i] = accC[i] = make_float2(0.f, 0.f);
        }
      }
    }
  };

  constexpr bool EARLY_REFILL = (MODE == 1 || MODE == 2);
  int it = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
    const int s = it % nstages;
    const uint32_t parity = (uint32_t)((it / nstages) & 1);
    Stage st{smem + s * stage_bytes, a.qbase};
    const int rows = (int)min((int64_t)TR, a.n - (int64_t)t * TR);
    const int rt = rows & ~7;
    if (!mbar_wait_bounded(&bars[s], parity)) s_err = 1;
    __syncthreads();
    if (s_err) break;
    // FP32-pipe dot forms with two or more stages: the stage consumed in the
    // previous iteration is refilled here, since the barrier above already
    // ordered every thread's last use of it, so the tile loop needs no
    // barrier at its end.  (The exact FP64 form keeps the refill at the end:
    // there the early one costs registers and occupancy.)
    if (EARLY_REFILL && nstages > 1 && tid == 0 && it > 0) {
      const int tn = t + (nstages - 1) * (int)gridDim.x;
      if (tn < a.ntiles) {
        const int sp = (it - 1) % nstages;
        fence_proxy_async();
        issue_tile<QT>(a, Stage{smem + sp * stage_bytes, a.qbase}, tn, &bars[sp]);
      }
    }
    if (tid >= rt && tid < rows) load_tail_row<QT>(a, st, t, tid);
    if (tid < rows) {
      if constexpr (MODE == 3) {
        uint64_t cv[2];
        row_program_dd(a, st, t, tid, co, cf, cv);
        for (int c = 0; c < a.ncol; ++c) {
          const uint64_t bit = 1ull << (c & 63);
          if ((a.dotcols[c >> 6] & bit) && !(cv[c >> 6] & bit)) st.put(c, tid, d2f2(st.d(c)[tid]));
        }
      } else if constexpr (MODE == 2) {
        double dv0 = 0.0, dv1 = 0.0;
        row_program_lp<QT>(a, st, t, tid, co, cf, (uint32_t)s_split[0], s_tymask, dv0, dv1);
#pragma unroll
        for (int d = 0; d < NRD; ++d) {
          if (d < dbase) {
            // FP64 columns 0, 1 are the row program's dv0, dv1; history
            // entries are read from the stage and converted exactly
            const int ca = sda[d], cb = sdb[d];
            const double va = ca >= a.qbase ? to_d<QT>(st.q<QT>(ca)[tid]) : (ca ? dv1 : dv0);
            const double vb = cb >= a.qbase ? to_d<QT>(st.q<QT>(cb)[tid]) : (cb ? dv1 : dv0);
            racc[d] = fma(va, vb, racc[d]);
          }
        }
      } else {
        row_program<QT>(a, st, t, tid, co);
        if constexpr (MODE == 1) {
          // FP64 squared norms, then the columns that feed the FP32-pipe
          // dot phase as scaled (hi, lo) floats (in place)
#pragma unroll
          for (int d = 0; d < NRD; ++d) {
            if (d < dbase) {
              const double v = st.d(a.dot_a[d])[tid];
              racc[d] = fma(v, v, racc[d]);
            }
          }
          for (int c = 0; c < a.ncol; ++c)
            if ((s_split[c >> 6] >> (c & 63)) & 1ull)
              st.put(c, tid, d2f2_dot(st.d(c)[tid], s_sb[c], s_lim[c]));
        }
      }
    }
    if constexpr (MODE == 0) {
      if (rowdots && tid < rows) {
#pragma unroll
        for (int d = 0; d < NRD; ++d) {
          if (d < a.ndots) {
            const int ca = sda[d], cb = sdb[d];
            racc[d] = fma(ldv<QT>(st, ca, tid, ca >= a.qbase), ldv<QT>(st, cb, tid, cb >= a.qbase),
                          racc[d]);
          }
        }
      }
    }
    if (!rowdots) __syncthreads();
    if constexpr (MODE == 2 && NSLOT == FAM_SLOTS) {
      if (famon && ncw > 0) {
        const int v0 = s_fam[3], v1 = s_fam[4], vq = s_fam[5];
        if (s_fam[1] == 2) {
          if (s_fam[2]) fam_tile<QT, 2, true>(st, fcol, ncw, v0, v1, vq, rows, lane, accS, accC);
          else fam_tile<QT, 2, false>(st, fcol, ncw, v0, v1, vq, rows, lane, accS, accC);
        } else {
          if (s_fam[2]) fam_tile<QT, 1, true>(st, fcol, ncw, v0, v1, vq, rows, lane, accS, accC);
          else fam_tile<QT, 1, false>(st, fcol, ncw, v0, v1, vq, rows, lane, accS, accC);
        }
      }
    }
    // dot phase: warp w owns dots w, w + NWARP, ...
#pragma unroll
    for (int i = 0; i < DPW; ++i) {
      if (rowdots || famon) break;
      const int d = dbase + warp + NWARP * i;
      if (d < a.ndots) {
        const int ca = sda[d], cb = sdb[d];
        if constexpr (MODE == 0) {
          const bool qa = ca >= a.qbase, qb = cb >= a.qbase;
          double sum = acc[i];
          for (int r = lane; r < rows; r += 32)
            sum = fma(ldv<QT>(st, ca, r, qa), ldv<QT>(st, cb, r, qb), sum);
          acc[i] = sum;
        } else {
          dot_tile<QT, MODE>(st, ca, cb, a.qbase, rows, lane, accS[i], accC[i]);
        }
      }
    }
    if constexpr (MODE != 0) {
      if ((it + 1) % FLUSH == 0) fold_slots(true);
    }
    if (!EARLY_REFILL || nstages == 1) {
      __syncthreads();
      if (tid == 0) {
        const int tn = t + (EARLY_REFILL ? 1 : nstages) * (int)gridDim.x;
        if (tn < a.ntiles) {
          fence_proxy_async();
          issue_tile<QT>(a, st, tn, &bars[s]);
        }
      }
    }
  }
  if constexpr (MODE != 0) fold_slots(false);

  const bool has_epilogue = a.ndots > 0 || a.kind == K_A || a.kind == K_PROJ;
  if (s_err) {
    // A copy did not complete in time: record it and give the copies still
    // in flight a bounded chance to land.  This CTA's partial sums are
    // unknown, so it posts NaN for every dot product and still takes its
    // ticket: the last CTA then finishes the reduction (NaN results), leaves
    // the m x m state untouched and resets the ticket for the next launch.
    if (tid == 0) {
      atomicExch(&S->st.status, DEV_ETIMEOUT);
      for (int s = 0; s < nstages; ++s) (void)mbar_wait_bounded(&bars[s], 0);
    }
    if (!has_epilogue) return;
    for (int d = tid; d < a.ndots; d += NT)
      a.partials[(size_t)blockIdx.x * NDOT_MAX + d] = __longlong_as_double(0x7ff8000000000000LL);
  }
  if (!has_epilogue) return;

  // Per-CTA partial sums (warp butterfly, then warps in order: fixed order).
  if (s_err) {
    // (NaN partials posted above)
  } else if (rowdots || MODE == 1 || MODE == 2) {
    const int nrow = (MODE == 1 || MODE == 2) ? dbase : a.ndots;
    __shared__ double rdw[NWARP][RD];
#pragma unroll
    for (int d = 0; d < NRD; ++d) {
      double v = racc[d];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) rdw[warp][d] = v;
    }
    __syncthreads();
    if (tid < nrow) {
      double v = 0.0;
      for (int w = 0; w < NWARP; ++w) v += rdw[w][tid];
      a.partials[(size_t)blockIdx.x * NDOT_MAX + tid] = v;
    }
  }
  if (!rowdots && !s_err) {
#pragma unroll
    for (int i = 0; i < NSLOT; ++i) {
      const int d = slot_dot(i);
      double v;
      if constexpr (SACC) {
        v = s_acc[warp][i];  // lane 0 wrote it and reads it below
      } else {
        v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      }
      if (lane == 0 && d < a.ndots) {
        if constexpr (MODE == 1) v *= pow2d(-(s_cexp[a.dot_a[d]] + s_cexp[a.dot_b[d]]));
        a.partials[(size_t)blockIdx.x * NDOT_MAX + d] = v;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned tk = atomicAdd(&S->ticket, 1u);
    s_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // Last CTA: finish the reduction.  Warp w owns dots w, w + NWARP, ...;
  // lane l sums the partials of CTAs l, l + 32, ... and a fixed butterfly
  // combines the lanes (bit-reproducible).
  for (int d = warp; d < a.ndots; d += NWARP) {
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(&a.partials[(size_t)b * NDOT_MAX + d]);
    v = warp_sum(v);
    if (lane == 0) S->red[d] = v;
  }
  __threadfence();
  __syncthreads();
  if (warp == 0) {
    // After a timed-out copy anywhere in the grid the sums are NaN: a plain
    // multi-dot still publishes them (NaN marks the failure for callers that
    // cannot read the status word); the m x m state is left as it was.
    const bool timed_out = *(volatile int32_t *)&S->st.status == DEV_ETIMEOUT;
    if (!timed_out || a.kind == K_MDOT) epilogue(a, (double *)smem, lane);
    if (lane == 0) S->ticket = 0;
    __threadfence();
  }
}

// ------------------------------------------------------------ host launch

template <class QT, int DPW, int MODE>
static cudaError_t launch_t(const PassArgs &a, int grid, size_t smem, int nstages,
                            cudaStream_t stream) {
  static bool attr_set = false;  // per instantiation
  auto kern = pass_kernel<QT, DPW, MODE>;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024 - 8 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  kern<<<grid, NT, smem, stream>>>(a, nstages);
  return cudaGetLastError();
}

template <class QT, int DPW, int MODE>
static int occupancy_t(size_t smem) {
  // resident CTAs per SM for this instantiation and dynamic shared memory
  // size, cached per host thread (the query sits on every pass launch)
  thread_local size_t key[32];
  thread_local int val[32];
  thread_local int used = 0;
  for (int i = 0; i < used; ++i)
    if (key[i] == smem) return val[i];
  int nb = 0;
  auto kern = pass_kernel<QT, DPW, MODE>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 8 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem) != cudaSuccess) return 1;
  nb = nb < 1 ? 1 : nb;
  if (used < 32) {
    key[used] = smem;
    val[used++] = nb;
  }
  return nb;
}

// Tile pipeline depth and grid of one pass.  The deepest pipeline (up to
// STAGES tiles in flight per CTA) that keeps the resident CTAs per SM at
// min(one-stage occupancy, 4): several CTAs at different points of their
// tile loop overlap copies with compute as well, and more of them overlap
// the FP64 row programs of some with the FP32-pipe dot phases of others,
// while more stages keep more bytes in flight per SM.  The first pass of the
// exact FP64 form, bound by the FP64 pipe, keeps two stages whenever they fit.
// (Measured at n = 406^3 for m = 5, 10, 20, 50.)
template <class QT, int DPW, int MODE>
static cudaError_t launch_shape(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  const size_t stage = stage_size<QT>(a);
  const size_t budget = 227 * 1024 - 8 * 1024;
  const size_t epi = epi_doubles(a.m > 0 ? a.m : 1) * sizeof(double);
  auto smem_for = [&](int ns) { return ns * stage < epi ? epi : ns * stage; };
  if (smem_for(1) > budget) return cudaErrorInvalidConfiguration;
  const int occ1 = occupancy_t<QT, DPW, MODE>(smem_for(1));
  const int want = occ1 < 4 ? occ1 : 4;
  int nstages = 1, occ = occ1;
  for (int ns = 2; ns <= STAGES; ++ns) {
    if (smem_for(ns) > budget) break;
    const int o = occupancy_t<QT, DPW, MODE>(smem_for(ns));
    const bool fp64_first = (MODE == 0 && a.kind == K_A && ns == 2);
    if (o >= want || fp64_first) {
      nstages = ns;
      occ = o;
    }
  }
  int grid = nsm * occ;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  return launch_t<QT, DPW, MODE>(a, grid, smem_for(nstages), nstages, stream);
}

template <class QT, int MODE>
static inline cudaError_t launch_qm(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  const int dpw_need = (a.ndots + NWARP - 1) / NWARP;
  if (dpw_need <= 1) return launch_shape<QT, 1, MODE>(a, nsm, grid_out, stream);
  if (dpw_need <= 4) return launch_shape<QT, 4, MODE>(a, nsm, grid_out, stream);
  if constexpr (MODE != 0) {
    // an exact bucket for up to 8 dots per warp (m = 20 ICWY: 56)
    if (dpw_need <= 8) return launch_shape<QT, 8, MODE>(a, nsm, grid_out, stream);
  }
  if (dpw_need <= 16) return launch_shape<QT, 16, MODE>(a, nsm, grid_out, stream);
  return launch_shape<QT, 32, MODE>(a, nsm, grid_out, stream);
}

}  // namespace aa
