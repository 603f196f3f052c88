// aa_common.h -- definitions shared by the host orchestration (aa_api.cu)
// and the streaming-pass kernels (aa_passes.cu).
//
// Every Anderson iteration is a short sequence of "streaming passes" over
// the n rows of the history.  A pass stages a tile of TR rows of a list of
// columns (history slots and FP64 vectors) into shared memory with bulk
// asynchronous copies, runs a per-row program (residual differences,
// Givens rotations, projections, the x update), and accumulates a list of
// dot products over the tile.  Per-CTA partial sums are finished by the last
// CTA to arrive, in a fixed order (bit-reproducible), which then runs the
// small m x m step of the algorithm (R, T, gamma) on the device.
#pragma once
#include <stdint.h>

namespace aa {

constexpr int TR = 256;                 // rows per tile (== threads per CTA)
constexpr int NT = 256;                 // threads per CTA
constexpr int NWARP = NT / 32;
constexpr int MMAX = 64;                // largest history depth
constexpr int MAXCOL = MMAX + 6;        // most columns one pass stages
constexpr int NDOT_MAX = 256;           // most dot products one pass reduces
constexpr int STAGES = 3;               // deepest tile pipeline (tiles in flight per CTA)

// Pass kinds.
enum PassKind : int {
  K_INIT = 0,    // first step: f0 = g0 - x0, x1 = g0
  K_A = 1,       // differences + QRDelete rotation + first reduction block
  K_PROJ = 2,    // v = w - Q coef (+ DCGS-2 correction of q_{k-1}); ||v||, v.f
  K_CGS2B = 3,   // CGS-2 middle pass: y = w - Q s; z = Q^T y
  K_MGS = 4,     // one MGS link: v -= r_{j-1} q_{j-1}; r_j = q_j^T v
  K_UPDATE = 5,  // x_{i+1} = g_i - dG gamma
  K_LSQ = 6,     // rhs = Q^T f, back-solve (unit API)
  K_MDOT = 7,    // plain multi-dot (unit API)
};

enum Orth : int { O_MGS = 0, O_ICWY = 1, O_CGS2 = 2, O_DCGS2 = 3 };

// Status words written by the device (first member of DevState so that the
// host reads them back with one small copy).
struct DevStatus {
  double fnorm2;     // ||f_i||^2 of the last K_A / K_INIT
  double dfnorm2;    // ||Delta f||^2 of the last K_A
  double rho;        // last new-column norm
  double xdiff2;     // ||x_{i+1} - x_i||^2 (stop rule 1)
  int32_t status;    // 0 or a negative AA_E* code raised on the device
  int32_t breakdown; // 1 if the last QRAdd broke down
  int32_t cols;      // columns held after the last completed QRAdd
  int32_t pad;
};

// Device-resident state of one context (m x m algebra lives here).
struct DevState {
  DevStatus st;
  double R[MMAX * MMAX];   // upper triangular, row-major, leading dimension MMAX
  double T[MMAX * MMAX];   // ICWY unit-lower correction I + L
  double Rn[MMAX * MMAX];  // R after the pending QRDelete
  double Tn[MMAX * MMAX];  // T after the pending QRDelete (ICWY, rotated at m x m level)
  double rot[4 * MMAX];    // folded rotation coefficients of the pending QRDelete
  double rot0;             // scale of stored column 0 (carry initialisation)
  double sig[MMAX];        // column scales: q_j = sig_j * u_j (u_j stored)
  double rhs[MMAX];        // Q^T f_i
  double coef[MMAX];       // projection coefficients folded with sig (next pass)
  double coef2[MMAX];      // DCGS-2 correction coefficients for q_{k-1}
  double s[MMAX];          // CGS-2 first-pass coefficients / DCGS-2 reorth coefficients
  double rcol[MMAX];       // R column under construction
  double gam[MMAX];        // gamma, logical order
  double gphys[MMAX];      // gamma in dG physical slot order (zeros elsewhere)
  double red[NDOT_MAX];    // result of the last reduction
  double vscale;           // stored new column = v * vscale
  double rcself;           // DCGS-2: scale applied to u_{k-1} in its correction
  int32_t pend_del;        // Rn/Tn/rot valid for the next QRDelete
  int32_t reorth;          // DCGS-2 correction active in the current add
  uint32_t ticket;         // last-CTA ticket (reset by the last CTA)
  int32_t pad;
};

// One launch of the streaming-pass kernel.
struct PassArgs {
  int kind;
  int orth;
  int64_t n;
  int ntiles;
  int ncol;                        // columns staged per tile
  int qbase;                       // first history column in the tile list
  int ndots;
  const void *col[MAXCOL];         // base pointers (tile t starts at col + t*TR)
  uint8_t pslot[MMAX];             // K_UPDATE: dG physical slot of tile column qbase + i
  uint8_t dot_a[NDOT_MAX];         // dot d = sum_r tile[a][r] * tile[b][r]
  uint8_t dot_b[NDOT_MAX];
  uint64_t dotcols[2];             // bit c: tile column c appears in a dot product
  // outputs (NULL when unused)
  void *out_q0;                    // history slot 0 written by the row program
  int64_t qstride;                 // bytes from one history slot to the next
  void *out_dg;                    // dG slot for Delta g (K_A step mode)
  double *out_df;                  // Delta f / y / v work vector (FP64)
  double *out_f;                   // f_i (overwrites f_{i-1})
  double *out_g;                   // g_i (overwrites g_{i-1})
  double *out_x;                   // x_{i+1}
  // shape of the add
  int m, c, k, del, step_mode;     // step_mode 1: AA step, 0: unit QRAdd / LSQ / MDOT
  int j0;                          // K_PROJ: first projected column (MGS: k-1)
  int jm;                          // K_MGS: link index j
  int ng;                          // K_UPDATE: dG columns in the tile
  int head_new;                    // dG ring head after this step
  int stop_kind;
  uint32_t flags;
  int dcgs2_min_mi;
  double breakdown_tol;
  int off_rhs, off_r, off_t, off_s, off_gram;  // offsets into the reduction result
  DevState *st;
  double *partials;                // [grid][NDOT_MAX]
  double *result_host_dev;         // K_MDOT: where the finished sums go (device)
};

}  // namespace aa
