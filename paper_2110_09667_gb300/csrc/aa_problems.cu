// aa_problems.cu -- built-in fixed-point maps G for the seeded stencil
// workloads, exported with the aa_g_fn signature so that aa_solve can run
// them without leaving C.  One thread per grid point; x fastest in memory;
// a 2D/3D launch so that no thread divides to find its coordinates.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/aa.h"

namespace {

// Launch shape: 32 threads along x (coalesced rows), 4 rows of y per block,
// one block row per (y block, z plane) of the grid: no index divisions.
constexpr int BX = 32, BY = 4;

// 2D anisotropic 5-point Jacobi: d = 2 + 2 eps, x neighbours -1, y
// neighbours -eps, zero Dirichlet boundary.  G(x) = x + D^{-1}(b - A x),
// evaluated with the diagonal term cancelled:
//   G = (b + (w + e) + eps (s + n)) / d   (rd = 1/d from the host).
__global__ void jacobi2d_kernel(const double *__restrict__ x, double *__restrict__ gx,
                                const double *__restrict__ b, int nx, int ny, double eps,
                                double rd) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int64_t p = (int64_t)j * nx + i;
  const double w = i > 0 ? x[p - 1] : 0.0;
  const double e = i < nx - 1 ? x[p + 1] : 0.0;
  const double s = j > 0 ? x[p - nx] : 0.0;
  const double n = j < ny - 1 ? x[p + nx] : 0.0;
  gx[p] = rd * (b[p] + fma(eps, s + n, w + e));
}

// 3D anisotropic 7-point weighted Jacobi: d = 2 (1 + ey + ez).
// G = x + omega D^{-1}(b - A x) with the diagonal term cancelled:
//   G = (1 - omega) x + (omega / d) (b + (w + e) + ey (s + n) + ez (dn + up)),
// eight FP64 operations per point (c0 = 1 - omega, c1 = omega / d).
__global__ void jacobi3d_kernel(const double *__restrict__ x, double *__restrict__ gx,
                                const double *__restrict__ b, int nx, int ny, int nz,
                                double ey, double ez, double c0, double c1) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= nx || j >= ny) return;
  const int64_t sxy = (int64_t)nx * ny;
  const int64_t p = (int64_t)k * sxy + (int64_t)j * nx + i;
  const double w = i > 0 ? x[p - 1] : 0.0;
  const double e = i < nx - 1 ? x[p + 1] : 0.0;
  const double s = j > 0 ? x[p - nx] : 0.0;
  const double n = j < ny - 1 ? x[p + nx] : 0.0;
  const double dn = k > 0 ? x[p - sxy] : 0.0;
  const double up = k < nz - 1 ? x[p + sxy] : 0.0;
  const double t = b[p] + fma(ez, dn + up, fma(ey, s + n, w + e));
  gx[p] = fma(c1, t, c0 * x[p]);
}

// Bratu nonlinear Jacobi on an s x s grid, h = 1/(s+1):
// G(u) = (sum of neighbours + h^2 (lambda e^u + src)) / 4  (h2 from the host).
__global__ void bratu2d_kernel(const double *__restrict__ u, double *__restrict__ gu,
                               const double *__restrict__ src, int s, double lambda, double h2) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= s || j >= s) return;
  const int64_t p = (int64_t)j * s + i;
  const double w = i > 0 ? u[p - 1] : 0.0;
  const double e = i < s - 1 ? u[p + 1] : 0.0;
  const double so = j > 0 ? u[p - s] : 0.0;
  const double no = j < s - 1 ? u[p + s] : 0.0;
  const double rhs = lambda * exp(u[p]) + (src ? src[p] : 0.0);
  gu[p] = ((w + e) + (so + no) + h2 * rhs) * 0.25;
}

dim3 grid2(int64_t nx, int64_t ny, int64_t nz) {
  return dim3((unsigned)((nx + BX - 1) / BX), (unsigned)((ny + BY - 1) / BY), (unsigned)nz);
}

// Grid extents the launch shape takes (x blocks unbounded in practice, y
// blocks and z planes at most 65535); larger problems are refused.
bool fits(int64_t nx, int64_t ny, int64_t nz) {
  return nx >= 1 && ny >= 1 && nz >= 1 && nx < (1LL << 31) && (ny + BY - 1) / BY <= 65535 &&
         nz <= 65535;
}

}  // namespace

extern "C" int aa_g_jacobi2d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_jacobi2d *P = (const aa_jacobi2d *)user;
  if (!P || !x || !gx || n != P->nx * P->ny || !fits(P->nx, P->ny, 1)) return AA_EINVAL;
  const double rd = 1.0 / (2.0 + 2.0 * P->eps);
  jacobi2d_kernel<<<grid2(P->nx, P->ny, 1), dim3(BX, BY), 0, (cudaStream_t)stream>>>(
      x, gx, P->b_dev, (int)P->nx, (int)P->ny, P->eps, rd);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_g_jacobi3d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_jacobi3d *P = (const aa_jacobi3d *)user;
  if (!P || !x || !gx || n != P->nx * P->ny * P->nz || !fits(P->nx, P->ny, P->nz))
    return AA_EINVAL;
  const double d = 2.0 * (1.0 + P->ey + P->ez);
  jacobi3d_kernel<<<grid2(P->nx, P->ny, P->nz), dim3(BX, BY), 0, (cudaStream_t)stream>>>(
      x, gx, P->b_dev, (int)P->nx, (int)P->ny, (int)P->nz, P->ey, P->ez, 1.0 - P->omega,
      P->omega / d);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_g_bratu2d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_bratu2d *P = (const aa_bratu2d *)user;
  if (!P || !x || !gx || n != P->s * P->s || !fits(P->s, P->s, 1)) return AA_EINVAL;
  const double h = 1.0 / (double)(P->s + 1);
  bratu2d_kernel<<<grid2(P->s, P->s, 1), dim3(BX, BY), 0, (cudaStream_t)stream>>>(
      x, gx, P->src_dev, (int)P->s, P->lambda, h * h);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}
