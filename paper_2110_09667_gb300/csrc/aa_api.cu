// aa_api.cu -- C ABI and host orchestration of the Anderson-acceleration
// passes (Algorithms 1 and 2 of the paper, QRAdd variants of Algorithms 3-6).
//
// The host keeps only what decides which passes to launch (column count,
// dG ring head, iteration index); every vector operation and every m x m
// step runs on the device (aa_passes.cu).  Per AA iteration at a full
// history the passes are:
//   MGS    : A (rotate + r_0), k-1 chained MGS links, PROJ, UPDATE
//   ICWY   : A (rotate + delayed T row + R column), PROJ, UPDATE
//   CGS-2  : A (rotate + s), CGS2B (y, z), PROJ, UPDATE
//   DCGS-2 : A (rotate + R column + reorth coefficients), PROJ (reorth of
//            q_{k-1} + projection), UPDATE
// with one grid-wide reduction per pass except UPDATE.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "../../include/aa.h"
#include "aa_common.h"

namespace aa {
cudaError_t launch_pass(const PassArgs &a, int storage, int nsm, int *grid_out,
                        cudaStream_t stream);
int max_grid(int nsm);
}  // namespace aa

using namespace aa;

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(x)                                                                 \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess)                                                          \
      return fail(AA_ECUDA, "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                              \
  } while (0)

struct aa_ctx {
  aa_config cfg;
  int64_t n, ld;
  int m, esz, nsm;
  cudaStream_t stream;
  char *Q, *dG;             // history storage: slot j at base + j*ld*esz
  double *DF, *fprev, *gprev;
  double *xbuf[2], *gbuf;   // aa_solve scratch (allocated on first use)
  DevState *st;
  double *partials;
  DevStatus *hstat;         // pinned
  double *hvec;             // pinned, MMAX doubles
  int c, head;
  int pend_k, pend_head;    // aa_step: the add in flight between launch and finish
  int64_t it;
  int need_reset;           // a device-reported error left the history undefined
  aa_stats stats;
  cudaEvent_t ev[4];
  // AA_FLAG_TIMING: event pairs around each pass, folded into per-kind sums
  // whenever the stream is synchronised.
  cudaEvent_t tev[2 * 256];
  int tkind[256];
  int tn;
  double pass_ms[8];
  int64_t pass_n[8];
};

extern "C" const char *aa_last_error(void) { return g_err.c_str(); }

extern "C" const char *aa_strerror(int code) {
  switch (code) {
    case AA_OK: return "ok";
    case AA_NOTCONVERGED: return "not converged";
    case AA_EINVAL: return "invalid argument";
    case AA_ENOMEM: return "out of memory";
    case AA_ECUDA: return "CUDA error";
    case AA_EBREAKDOWN: return "QR update breakdown (history cleared)";
    case AA_ENONFINITE: return "non-finite residual";
    case AA_ETIMEOUT: return "device wait timed out";
    case AA_ECALLBACK: return "G callback failed";
    case AA_ESTATE: return "invalid state";
    default: return "unknown";
  }
}

extern "C" const char *aa_version(void) { return "libaa 0.1 sm_103a"; }

extern "C" void aa_config_default(aa_config *cfg, int64_t n) {
  memset(cfg, 0, sizeof *cfg);
  cfg->n = n;
  cfg->m = 5;
  cfg->orth = AA_MGS;
  cfg->storage = AA_STORE_FP64;
  cfg->max_iters = 100;
  cfg->tol = 1e-8;
  cfg->scale = 1.0;
  cfg->stop_kind = 0;
  cfg->dcgs2_min_mi = 3;
  cfg->breakdown_tol = 1e-14;
  cfg->flags = 0;
  cfg->stream = nullptr;
}

static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" int aa_create(const aa_config *cfg, aa_ctx **out) {
  if (!cfg || !out) return fail(AA_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->n < 1) return fail(AA_EINVAL, "n must be >= 1");
  if (cfg->m < 1 || cfg->m > MMAX) return fail(AA_EINVAL, "m must be in 1..%d", MMAX);
  if (cfg->orth < 0 || cfg->orth > 3) return fail(AA_EINVAL, "bad orth");
  if (cfg->storage < 0 || cfg->storage > 2) return fail(AA_EINVAL, "bad storage");
  if (cfg->stop_kind < 0 || cfg->stop_kind > 1) return fail(AA_EINVAL, "bad stop_kind");
  if (!(cfg->scale > 0)) return fail(AA_EINVAL, "scale must be > 0");
  if ((cfg->flags & AA_FLAG_ICWY_GRAM) && cfg->m > 24)
    return fail(AA_EINVAL, "AA_FLAG_ICWY_GRAM needs m <= 24");
  if ((cfg->flags & AA_FLAG_DF_ARITH) &&
      ((cfg->flags & AA_FLAG_FP32_DOTS) || cfg->storage != AA_STORE_FP64))
    return fail(AA_EINVAL, "AA_FLAG_DF_ARITH needs FP64 storage and no AA_FLAG_FP32_DOTS");
  if (cfg->n > (int64_t)2147483647 * TR) return fail(AA_EINVAL, "n too large");
  aa_ctx *c = (aa_ctx *)calloc(1, sizeof(aa_ctx));
  if (!c) return fail(AA_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  if (c->cfg.breakdown_tol <= 0) c->cfg.breakdown_tol = 1e-14;
  c->n = cfg->n;
  c->m = cfg->m;
  c->esz = cfg->storage == AA_STORE_FP64 ? 8 : (cfg->storage == AA_STORE_FP32 ? 4 : 2);
  c->ld = round_up(cfg->n, 128);  // every slot starts 256-byte aligned
  c->stream = (cudaStream_t)cfg->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (c->nsm < 1) c->nsm = 1;
  auto cleanup = [&](int code) {
    aa_destroy(c);
    return code;
  };
  const size_t hist = (size_t)c->ld * c->m * c->esz;
  if (cudaMalloc(&c->Q, hist) != cudaSuccess || cudaMalloc(&c->dG, hist) != cudaSuccess ||
      cudaMalloc(&c->DF, (size_t)c->ld * 8) != cudaSuccess ||
      cudaMalloc(&c->fprev, (size_t)c->ld * 8) != cudaSuccess ||
      cudaMalloc(&c->gprev, (size_t)c->ld * 8) != cudaSuccess ||
      cudaMalloc(&c->st, sizeof(DevState)) != cudaSuccess ||
      cudaMalloc(&c->partials, (size_t)max_grid(c->nsm) * NDOT_MAX * 8) != cudaSuccess ||
      cudaMallocHost(&c->hstat, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->hvec, MMAX * 8) != cudaSuccess) {
    cudaGetLastError();
    fail(AA_ENOMEM, "device allocation of %.2f GB failed", (2.0 * hist + 3.0 * c->ld * 8) / 1e9);
    return cleanup(AA_ENOMEM);
  }
  if (cudaMemset(c->Q, 0, hist) != cudaSuccess || cudaMemset(c->dG, 0, hist) != cudaSuccess ||
      cudaMemset(c->st, 0, sizeof(DevState)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    fail(AA_ECUDA, "initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    return cleanup(AA_ECUDA);
  }
  for (int i = 0; i < 4; ++i) cudaEventCreate(&c->ev[i]);
  if (c->cfg.flags & AA_FLAG_TIMING)
    for (int i = 0; i < 2 * 256; ++i) cudaEventCreate(&c->tev[i]);
  *out = c;
  return AA_OK;
}

extern "C" void aa_destroy(aa_ctx *c) {
  if (!c) return;
  if (c->stream || c->Q) cudaStreamSynchronize(c->stream);
  cudaFree(c->Q);
  cudaFree(c->dG);
  cudaFree(c->DF);
  cudaFree(c->fprev);
  cudaFree(c->gprev);
  cudaFree(c->xbuf[0]);
  cudaFree(c->xbuf[1]);
  cudaFree(c->gbuf);
  cudaFree(c->st);
  cudaFree(c->partials);
  if (c->hstat) cudaFreeHost(c->hstat);
  if (c->hvec) cudaFreeHost(c->hvec);
  for (int i = 0; i < 4; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (int i = 0; i < 2 * 256; ++i)
    if (c->tev[i]) cudaEventDestroy(c->tev[i]);
  free(c);
}

extern "C" int aa_reset(aa_ctx *c) {
  if (!c) return fail(AA_EINVAL, "NULL ctx");
  c->c = 0;
  c->head = 0;
  c->it = 0;
  memset(&c->stats, 0, sizeof c->stats);
  memset(c->pass_ms, 0, sizeof c->pass_ms);
  memset(c->pass_n, 0, sizeof c->pass_n);
  c->tn = 0;
  CUDA_TRY(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  c->need_reset = 0;
  return AA_OK;
}

// Calls that use the history refuse to run after a device-reported error
// (a pass that gave up on a bounded wait may have rotated part of Q; a
// non-finite residual cleared the history on the device but not on the
// host) until aa_reset starts a fresh history.
static int check_usable(aa_ctx *c) {
  if (c->need_reset)
    return fail(AA_ESTATE, "a device error left the history undefined: call aa_reset first");
  return AA_OK;
}

extern "C" int aa_test_set_device_status(aa_ctx *c, int code) {
  if (!c) return fail(AA_EINVAL, "NULL ctx");
  if (code > 0) return fail(AA_EINVAL, "status codes are 0 or negative");
  const int32_t v = code;
  CUDA_TRY(cudaMemcpyAsync(&c->st->st.status, &v, sizeof v, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return AA_OK;
}

extern "C" int aa_set_stream(aa_ctx *c, void *stream) {
  if (!c) return fail(AA_EINVAL, "NULL ctx");
  c->stream = (cudaStream_t)stream;
  c->cfg.stream = stream;
  return AA_OK;
}

extern "C" int aa_pass_times(const aa_ctx *c, double *ms_out, int64_t *count_out) {
  if (!c || !ms_out || !count_out) return fail(AA_EINVAL, "NULL argument");
  for (int k = 0; k < 8; ++k) {
    ms_out[k] = c->pass_ms[k];
    count_out[k] = c->pass_n[k];
  }
  return AA_OK;
}

extern "C" int aa_get_stats(const aa_ctx *c, aa_stats *out) {
  if (!c || !out) return fail(AA_EINVAL, "NULL argument");
  *out = c->stats;
  return AA_OK;
}

// ------------------------------------------------------------------ passes

static void *qslot(aa_ctx *c, int j) { return c->Q + (size_t)j * c->ld * c->esz; }
static void *gslot(aa_ctx *c, int p) { return c->dG + (size_t)p * c->ld * c->esz; }

static void base_args(aa_ctx *c, PassArgs &a, int kind) {
  memset(&a, 0, sizeof a);
  a.kind = kind;
  a.orth = c->cfg.orth;
  a.n = c->n;
  a.ntiles = (int)((c->n + TR - 1) / TR);
  a.m = c->m;
  a.flags = (uint32_t)c->cfg.flags;
  a.dcgs2_min_mi = c->cfg.dcgs2_min_mi;
  a.breakdown_tol = c->cfg.breakdown_tol;
  a.stop_kind = c->cfg.stop_kind;
  a.st = c->st;
  a.partials = c->partials;
  a.out_q0 = qslot(c, 0);
  a.qstride = c->ld * c->esz;
}

static void add_dot(PassArgs &a, int x, int y) {
  a.dot_a[a.ndots] = (uint8_t)x;
  a.dot_b[a.ndots] = (uint8_t)y;
  a.dotcols[x >> 6] |= 1ull << (x & 63);
  a.dotcols[y >> 6] |= 1ull << (y & 63);
  a.ndots++;
}

// Fold recorded pass events into the per-kind sums (stream already synced).
static void fold_timing(aa_ctx *c) {
  for (int i = 0; i < c->tn; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->tev[2 * i], c->tev[2 * i + 1]) == cudaSuccess) {
      c->pass_ms[c->tkind[i]] += ms;
      c->pass_n[c->tkind[i]] += 1;
    }
  }
  c->tn = 0;
}

static int run(aa_ctx *c, const PassArgs &a) {
  int grid = 0;
  const bool timing = (c->cfg.flags & AA_FLAG_TIMING) && c->tev[0];
  if (timing && c->tn == 256) {
    cudaStreamSynchronize(c->stream);
    fold_timing(c);
  }
  if (timing) cudaEventRecord(c->tev[2 * c->tn], c->stream);
  cudaError_t e = launch_pass(a, c->cfg.storage, c->nsm, &grid, c->stream);
  if (timing && e == cudaSuccess) {
    cudaEventRecord(c->tev[2 * c->tn + 1], c->stream);
    c->tkind[c->tn++] = a.kind;
  }
  if (e != cudaSuccess) return fail(AA_ECUDA, "pass %d launch failed: %s", a.kind, cudaGetErrorString(e));
  c->stats.launches++;
  if (a.ndots > 0 && a.kind != K_UPDATE) c->stats.reductions++;
  return AA_OK;
}

// Does this add run the DCGS-2 correction of q_{k-1}?  (m_i = k + 1.)
static bool dcgs2_reorth(aa_ctx *c, int k) {
  return c->cfg.orth == AA_DCGS2 && (k + 1) > c->cfg.dcgs2_min_mi && k >= 2;
}

// First pass of an add: differences (step mode), QRDelete rotation when the
// history is full, and the first block of dot products.
static int pass_A(aa_ctx *c, bool step, const double *x, const double *g, const double *v,
                  int k, bool del, int dg_slot, int head_new) {
  PassArgs a;
  base_args(c, a, K_A);
  a.step_mode = step;
  a.head_new = head_new;
  a.c = c->c;
  a.k = k;
  a.del = del;
  if (dcgs2_reorth(c, k)) a.flags |= 0x100u;
  int nc = 0;
  if (step) {
    a.col[nc++] = x;
    a.col[nc++] = g;
    a.col[nc++] = c->gprev;
    a.col[nc++] = c->fprev;
    a.out_dg = gslot(c, dg_slot);
    a.out_f = c->fprev;
    a.out_g = c->gprev;
  } else {
    a.col[nc++] = v;
  }
  a.out_df = c->DF;
  a.qbase = nc;
  for (int j = 0; j < c->c; ++j) a.col[nc++] = qslot(c, j);
  a.ncol = nc;
  const int qb = a.qbase;
  // tile columns: step: 0 f, 1 df ; unit: 0 df
  const int cdf = step ? 1 : 0, cf = 0;
  if (step) {
    add_dot(a, cf, cf);
    add_dot(a, cdf, cdf);
    add_dot(a, cdf, cf);
  } else {
    add_dot(a, cdf, cdf);
  }
  if (k > 0) {
    if (step) {
      a.off_rhs = a.ndots;
      for (int j = 0; j < k; ++j) add_dot(a, qb + j, cf);
    }
    a.off_r = a.ndots;
    if (c->cfg.orth == AA_MGS) {
      add_dot(a, qb + 0, cdf);
    } else {
      for (int j = 0; j < k; ++j) add_dot(a, qb + j, cdf);
    }
    if (c->cfg.orth == AA_ICWY) {
      a.off_t = a.ndots;
      for (int l = 0; l + 1 < k; ++l) add_dot(a, qb + l, qb + k - 1);
      if ((c->cfg.flags & AA_FLAG_ICWY_GRAM) && del) {
        a.off_gram = a.ndots;
        for (int j = 1; j <= k - 2; ++j)
          for (int l = 0; l < j; ++l) add_dot(a, qb + l, qb + j);
      }
    }
    if (c->cfg.orth == AA_DCGS2 && dcgs2_reorth(c, k)) {
      a.off_s = a.ndots;
      for (int j = 0; j + 1 < k; ++j) add_dot(a, qb + j, qb + k - 1);
    }
  }
  if (a.ndots > NDOT_MAX) return fail(AA_EINVAL, "too many dot products (%d)", a.ndots);
  return run(c, a);
}

static int pass_mgs_link(aa_ctx *c, int k, int jm) {
  PassArgs a;
  base_args(c, a, K_MGS);
  a.k = k;
  a.jm = jm;
  a.col[0] = c->DF;
  a.qbase = 1;
  a.col[1] = qslot(c, jm - 1);
  a.col[2] = qslot(c, jm);
  a.ncol = 3;
  a.out_df = c->DF;
  add_dot(a, 2, 0);
  return run(c, a);
}

static int pass_cgs2b(aa_ctx *c, int k) {
  PassArgs a;
  base_args(c, a, K_CGS2B);
  a.k = k;
  a.col[0] = c->DF;
  a.qbase = 1;
  for (int j = 0; j < k; ++j) a.col[1 + j] = qslot(c, j);
  a.ncol = 1 + k;
  a.out_df = c->DF;
  for (int j = 0; j < k; ++j) add_dot(a, 1 + j, 0);
  return run(c, a);
}

static int pass_proj(aa_ctx *c, bool step, int k, int j0, int head_new) {
  PassArgs a;
  base_args(c, a, K_PROJ);
  a.step_mode = step;
  a.k = k;
  a.j0 = j0;
  a.head_new = head_new;
  const bool reorth = dcgs2_reorth(c, k);
  if (reorth) a.flags |= 0x100u;
  int nc = 0;
  a.col[nc++] = c->DF;
  if (step) a.col[nc++] = c->fprev;  // holds f_i after pass A
  a.qbase = nc;
  for (int j = j0; j < k; ++j) a.col[nc++] = qslot(c, j);
  a.ncol = nc;
  add_dot(a, 0, 0);
  if (step) {
    add_dot(a, 0, 1);
    if (reorth) add_dot(a, a.qbase + (k - 1 - j0), 1);
  }
  return run(c, a);
}

static int pass_update(aa_ctx *c, const double *g, const double *x, double *xn, int ng,
                       int head_new) {
  PassArgs a;
  base_args(c, a, K_UPDATE);
  int nc = 0;
  a.col[nc++] = g;
  if (c->cfg.stop_kind == 1) a.col[nc++] = x;
  a.qbase = nc;
  for (int i = 0; i < ng; ++i) {
    const int p = (head_new + i) % c->m;
    a.pslot[i] = (uint8_t)p;
    a.col[nc++] = gslot(c, p);
  }
  a.ncol = nc;
  a.ng = ng;
  a.out_x = xn;
  if (c->cfg.stop_kind == 1) add_dot(a, 1, 1);
  return run(c, a);
}

// The status word is read in two halves so that a caller can enqueue more
// work (a timing event) between the copy and the wait.
static int status_copy(aa_ctx *c) {
  CUDA_TRY(cudaMemcpyAsync(c->hstat, &c->st->st, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                           c->stream));
  return AA_OK;
}

static int status_wait(aa_ctx *c) {
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->tn) fold_timing(c);
  if (c->hstat->status != 0) {
    const int code = c->hstat->status;
    // clear the sticky device status and ticket so the context stays usable
    cudaMemsetAsync(&c->st->st.status, 0, sizeof(int32_t), c->stream);
    cudaMemsetAsync(&c->st->ticket, 0, sizeof(uint32_t), c->stream);
    cudaStreamSynchronize(c->stream);
    c->need_reset = 1;
    return fail(code, "device reported %s (history undefined until aa_reset)", aa_strerror(code));
  }
  return AA_OK;
}

static int read_status(aa_ctx *c) {
  int rc = status_copy(c);
  return rc ? rc : status_wait(c);
}

// The QR update of Algorithm 2 for one new column (step or unit mode).
// Leaves the device state with the new R column, and (step mode) gamma.
static int qr_update(aa_ctx *c, bool step, const double *x, const double *g, const double *v,
                     int *k_out, int *head_new_out, int *dg_slot_out) {
  const int m = c->m;
  const bool del = (c->c == m);
  const int k = del ? m - 1 : c->c;
  int head_new = c->head, dg_slot;
  if (del) {
    dg_slot = c->head;
    head_new = (c->head + 1) % m;
  } else {
    dg_slot = (c->head + c->c) % m;
  }
  int rc = pass_A(c, step, x, g, v, k, del, dg_slot, head_new);
  if (rc) return rc;
  if (k > 0) {
    switch (c->cfg.orth) {
      case AA_MGS:
        for (int j = 1; j < k; ++j)
          if ((rc = pass_mgs_link(c, k, j))) return rc;
        rc = pass_proj(c, step, k, k - 1, head_new);
        break;
      case AA_CGS2:
        if ((rc = pass_cgs2b(c, k))) return rc;
        rc = pass_proj(c, step, k, 0, head_new);
        break;
      default:
        rc = pass_proj(c, step, k, 0, head_new);
        break;
    }
    if (rc) return rc;
  }
  *k_out = k;
  *head_new_out = head_new;
  *dg_slot_out = dg_slot;
  return AA_OK;
}

// aa_step in two halves: step_launch enqueues the passes of one iteration
// and the copy of the status word; step_finish waits for them and updates the
// host-side history bookkeeping.  (aa_solve records a timing event between
// the two, so that it needs no second synchronisation.)
static int step_launch(aa_ctx *c, const double *x, const double *g, double *xn) {
  if (!c || !x || !g || !xn) return fail(AA_EINVAL, "NULL argument");
  if (!aligned16(x) || !aligned16(g) || !aligned16(xn))
    return fail(AA_EINVAL, "device vectors must be 16-byte aligned");
  if (xn == x || xn == g) return fail(AA_EINVAL, "xnext must not alias x or G(x)");
  int rc = check_usable(c);
  if (rc) return rc;
  if (c->it == 0) {
    PassArgs a;
    base_args(c, a, K_INIT);
    a.col[0] = x;
    a.col[1] = g;
    a.ncol = 2;
    a.qbase = 2;
    a.out_f = c->fprev;
    a.out_g = c->gprev;
    a.out_x = xn;
    add_dot(a, 0, 0);
    if ((rc = run(c, a))) return rc;
    return status_copy(c);
  }
  int k, head_new, dg_slot;
  if ((rc = qr_update(c, true, x, g, nullptr, &k, &head_new, &dg_slot))) return rc;
  if ((rc = pass_update(c, c->gprev, x, xn, k + 1, head_new))) return rc;
  c->pend_k = k;
  c->pend_head = head_new;
  return status_copy(c);
}

static int step_finish(aa_ctx *c, double *fnorm) {
  int rc;
  if ((rc = status_wait(c))) return rc;
  c->stats.steps++;
  c->stats.fnorm = sqrt(c->hstat->fnorm2);
  if (fnorm) *fnorm = c->stats.fnorm;
  if (c->it == 0) {
    c->it = 1;
    return AA_OK;
  }
  if (c->hstat->breakdown) {
    c->stats.breakdowns++;
    c->c = 0;
    c->head = 0;
  } else {
    c->c = c->pend_k + 1;
    c->head = c->pend_head;
  }
  c->it++;
  return AA_OK;
}

extern "C" int aa_step(aa_ctx *c, const double *x, const double *g, double *xn, double *fnorm) {
  int rc = step_launch(c, x, g, xn);
  return rc ? rc : step_finish(c, fnorm);
}

extern "C" int aa_qradd(aa_ctx *c, const double *v) {
  if (!c || !v) return fail(AA_EINVAL, "NULL argument");
  if (!aligned16(v)) return fail(AA_EINVAL, "v must be 16-byte aligned");
  if (check_usable(c)) return AA_ESTATE;
  int k, head_new, dg_slot;
  int rc = qr_update(c, false, nullptr, nullptr, v, &k, &head_new, &dg_slot);
  if (rc) return rc;
  if ((rc = read_status(c))) return rc;
  if (c->hstat->breakdown) {
    c->c = 0;
    c->head = 0;
    c->stats.breakdowns++;
    return fail(AA_EBREAKDOWN, "new column in span(Q): history cleared");
  }
  c->c = k + 1;
  c->head = head_new;
  return AA_OK;
}

extern "C" int aa_lsq(aa_ctx *c, const double *f, double *gamma_host) {
  if (!c || !f || !gamma_host) return fail(AA_EINVAL, "NULL argument");
  if (!aligned16(f)) return fail(AA_EINVAL, "f must be 16-byte aligned");
  if (check_usable(c)) return AA_ESTATE;
  if (c->c == 0) return 0;
  PassArgs a;
  base_args(c, a, K_LSQ);
  a.c = c->c;
  a.col[0] = f;
  a.qbase = 1;
  for (int j = 0; j < c->c; ++j) {
    a.col[1 + j] = qslot(c, j);
    add_dot(a, 1 + j, 0);
  }
  a.ncol = 1 + c->c;
  int rc = run(c, a);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(c->hvec, c->st->gam, sizeof(double) * c->c, cudaMemcpyDeviceToHost,
                           c->stream));
  if ((rc = read_status(c))) return rc;
  memcpy(gamma_host, c->hvec, sizeof(double) * c->c);
  return c->c;
}

extern "C" int aa_get_qr(aa_ctx *c, double *Qh, double *Rh, double *Th, int *k) {
  if (!c || !k) return fail(AA_EINVAL, "NULL argument");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int kc = c->c;
  *k = kc;
  DevState *hs = (DevState *)malloc(sizeof(DevState));
  if (!hs) return fail(AA_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpy(hs, c->st, sizeof(DevState), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(hs);
    return fail(AA_ECUDA, "state copy failed: %s", cudaGetErrorString(e));
  }
  if (Rh)
    for (int j = 0; j < kc; ++j)
      for (int l = 0; l < kc; ++l) Rh[j * kc + l] = hs->R[j * MMAX + l];
  if (Th)
    for (int j = 0; j < kc; ++j)
      for (int l = 0; l < kc; ++l) Th[j * kc + l] = hs->T[j * MMAX + l];
  if (Qh) {
    char *tmp = (char *)malloc((size_t)c->n * c->esz);
    if (!tmp) {
      free(hs);
      return fail(AA_ENOMEM, "host allocation failed");
    }
    for (int j = 0; j < kc; ++j) {
      e = cudaMemcpy(tmp, qslot(c, j), (size_t)c->n * c->esz, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        free(tmp);
        free(hs);
        return fail(AA_ECUDA, "Q copy failed: %s", cudaGetErrorString(e));
      }
      const double s = hs->sig[j];
      double *dst = Qh + (size_t)j * c->n;
      for (int64_t i = 0; i < c->n; ++i) {
        double u;
        if (c->esz == 8) {
          u = ((double *)tmp)[i];
        } else if (c->esz == 4) {
          u = (double)((float *)tmp)[i];
        } else {
          uint32_t b = (uint32_t)((uint16_t *)tmp)[i] << 16;
          float f;
          memcpy(&f, &b, 4);
          u = (double)f;
        }
        dst[i] = s * u;
      }
    }
    free(tmp);
  }
  free(hs);
  return AA_OK;
}

extern "C" int aa_solve(aa_ctx *c, aa_g_fn G, void *user, double *x, aa_stats *stats) {
  if (!c || !G || !x) return fail(AA_EINVAL, "NULL argument");
  if (!aligned16(x)) return fail(AA_EINVAL, "x must be 16-byte aligned");
  if (!c->xbuf[0]) {
    if (cudaMalloc(&c->xbuf[0], (size_t)c->ld * 8) != cudaSuccess ||
        cudaMalloc(&c->xbuf[1], (size_t)c->ld * 8) != cudaSuccess ||
        cudaMalloc(&c->gbuf, (size_t)c->ld * 8) != cudaSuccess) {
      cudaGetLastError();
      return fail(AA_ENOMEM, "solve buffers");
    }
  }
  int rc = aa_reset(c);
  if (rc) return rc;
  const double tol_abs = c->cfg.tol * c->cfg.scale;
  double *cur = x;
  int nb = 0;
  int status = AA_NOTCONVERGED;
  float gms = 0.f, ams = 0.f;
  int64_t i;
  for (i = 0;; ++i) {
    cudaEventRecord(c->ev[0], c->stream);
    if (G(cur, c->gbuf, c->n, (void *)c->stream, user) != 0) {
      status = fail(AA_ECALLBACK, "G callback returned an error at iteration %lld", (long long)i);
      break;
    }
    cudaEventRecord(c->ev[1], c->stream);
    double *nxt = c->xbuf[nb];
    double fn = 0;
    rc = step_launch(c, cur, c->gbuf, nxt);
    cudaEventRecord(c->ev[2], c->stream);
    if (rc == AA_OK) rc = step_finish(c, &fn);  // its wait covers the event too
    else cudaEventSynchronize(c->ev[2]);
    float t1 = 0, t2 = 0;
    cudaEventElapsedTime(&t1, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&t2, c->ev[1], c->ev[2]);
    gms += t1;
    ams += t2;
    if (rc) {
      status = rc;
      break;
    }
    if (c->cfg.stop_kind == 0 && fn < tol_abs) {
      status = AA_OK;
      break;
    }
    if (i == c->cfg.max_iters) break;
    if (c->cfg.stop_kind == 1 && sqrt(c->hstat->xdiff2) < c->cfg.tol) {
      cur = nxt;
      ++i;
      status = AA_OK;
      break;
    }
    cur = nxt;
    nb ^= 1;
  }
  if (cur != x) {
    cudaError_t e = cudaMemcpyAsync(x, cur, (size_t)c->n * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return fail(AA_ECUDA, "copy-out failed");
    cudaStreamSynchronize(c->stream);
  }
  c->stats.iters = i;
  c->stats.g_ms = gms;
  c->stats.aa_ms = ams;
  if (stats) *stats = c->stats;
  return status;
}

// ------------------------------------------------------------ aa_mdot

extern "C" int aa_mdot(const double *A, int64_t lda, int k, const double *V, int64_t ldv, int nv,
                       int64_t n, double *out_host, void *stream) {
  if (!A || !V || !out_host) return fail(AA_EINVAL, "NULL argument");
  if (n < 1 || k < 1 || nv < 1 || k * nv > NDOT_MAX || k + nv > MAXCOL || lda < n || ldv < n)
    return fail(AA_EINVAL, "bad sizes");
  for (int j = 0; j < k; ++j)
    if (!aligned16(A + (size_t)j * lda)) return fail(AA_EINVAL, "A columns must be 16-byte aligned");
  for (int v = 0; v < nv; ++v)
    if (!aligned16(V + (size_t)v * ldv)) return fail(AA_EINVAL, "V columns must be 16-byte aligned");
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = (cudaStream_t)stream;
  DevState *st = nullptr;
  double *partials = nullptr, *res = nullptr;
  int rc = AA_OK;
  if (cudaMalloc(&st, sizeof(DevState)) != cudaSuccess ||
      cudaMalloc(&partials, (size_t)aa::max_grid(nsm) * NDOT_MAX * 8) != cudaSuccess ||
      cudaMalloc(&res, NDOT_MAX * 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(st);
    cudaFree(partials);
    cudaFree(res);
    return fail(AA_ENOMEM, "scratch allocation failed");
  }
  PassArgs a;
  memset(&a, 0, sizeof a);
  a.kind = K_MDOT;
  a.n = n;
  a.ntiles = (int)((n + TR - 1) / TR);
  a.m = 1;
  for (int j = 0; j < k; ++j) a.col[j] = A + (size_t)j * lda;
  for (int v = 0; v < nv; ++v) a.col[k + v] = V + (size_t)v * ldv;
  a.ncol = k + nv;
  a.qbase = a.ncol;
  for (int j = 0; j < k; ++j)
    for (int v = 0; v < nv; ++v) add_dot(a, j, k + v);
  a.st = st;
  a.partials = partials;
  a.result_host_dev = res;
  int grid = 0;
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevState), s);
  if (e == cudaSuccess) e = launch_pass(a, 0, nsm, &grid, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, res, sizeof(double) * k * nv, cudaMemcpyDeviceToHost, s);
  int32_t dev_status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&dev_status, &st->st.status, sizeof dev_status, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = fail(AA_ECUDA, "aa_mdot: %s", cudaGetErrorString(e));
  else if (dev_status != 0) rc = fail(dev_status, "aa_mdot: device reported %s", aa_strerror(dev_status));
  cudaFree(st);
  cudaFree(partials);
  cudaFree(res);
  return rc;
}
