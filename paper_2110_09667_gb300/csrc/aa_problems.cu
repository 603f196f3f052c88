// aa_problems.cu -- built-in fixed-point maps G for the seeded stencil
// workloads, exported with the aa_g_fn signature so that aa_solve can run
// them without leaving C.  One thread per grid point; x fastest in memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/aa.h"

namespace {

// 2D anisotropic 5-point Jacobi: d = 2 + 2 eps, x neighbours -1, y
// neighbours -eps, zero Dirichlet boundary.  G(x) = x + D^{-1}(b - A x).
__global__ void jacobi2d_kernel(const double *__restrict__ x, double *__restrict__ gx,
                                const double *__restrict__ b, int64_t nx, int64_t ny, double eps) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny) return;
  const int64_t j = p / nx, i = p - j * nx;
  const double d = 2.0 + 2.0 * eps;
  const double w = i > 0 ? x[p - 1] : 0.0;
  const double e = i < nx - 1 ? x[p + 1] : 0.0;
  const double s = j > 0 ? x[p - nx] : 0.0;
  const double n = j < ny - 1 ? x[p + nx] : 0.0;
  const double ax = d * x[p] - (w + e) - eps * (s + n);
  gx[p] = x[p] + (b[p] - ax) / d;
}

// 3D anisotropic 7-point weighted Jacobi: d = 2 (1 + ey + ez).
__global__ void jacobi3d_kernel(const double *__restrict__ x, double *__restrict__ gx,
                                const double *__restrict__ b, int64_t nx, int64_t ny, int64_t nz,
                                double ey, double ez, double omega) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sxy = nx * ny;
  if (p >= sxy * nz) return;
  const int64_t k = p / sxy;
  const int64_t r = p - k * sxy;
  const int64_t j = r / nx, i = r - j * nx;
  const double d = 2.0 * (1.0 + ey + ez);
  const double w = i > 0 ? x[p - 1] : 0.0;
  const double e = i < nx - 1 ? x[p + 1] : 0.0;
  const double s = j > 0 ? x[p - nx] : 0.0;
  const double n = j < ny - 1 ? x[p + nx] : 0.0;
  const double dn = k > 0 ? x[p - sxy] : 0.0;
  const double up = k < nz - 1 ? x[p + sxy] : 0.0;
  const double ax = d * x[p] - (w + e) - ey * (s + n) - ez * (dn + up);
  gx[p] = x[p] + omega * (b[p] - ax) / d;
}

// Bratu nonlinear Jacobi on an s x s grid, h = 1/(s+1):
// G(u) = (sum of neighbours + h^2 (lambda e^u + src)) / 4.
__global__ void bratu2d_kernel(const double *__restrict__ u, double *__restrict__ gu,
                               const double *__restrict__ src, int64_t s, double lambda) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s * s) return;
  const int64_t j = p / s, i = p - j * s;
  const double h = 1.0 / (double)(s + 1);
  const double h2 = h * h;
  const double w = i > 0 ? u[p - 1] : 0.0;
  const double e = i < s - 1 ? u[p + 1] : 0.0;
  const double so = j > 0 ? u[p - s] : 0.0;
  const double no = j < s - 1 ? u[p + s] : 0.0;
  const double rhs = lambda * exp(u[p]) + (src ? src[p] : 0.0);
  gu[p] = ((w + e) + (so + no) + h2 * rhs) / 4.0;
}

int grid_for(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace

extern "C" int aa_g_jacobi2d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_jacobi2d *P = (const aa_jacobi2d *)user;
  if (!P || !x || !gx || n != P->nx * P->ny) return AA_EINVAL;
  jacobi2d_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, gx, P->b_dev, P->nx, P->ny,
                                                                 P->eps);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_g_jacobi3d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_jacobi3d *P = (const aa_jacobi3d *)user;
  if (!P || !x || !gx || n != P->nx * P->ny * P->nz) return AA_EINVAL;
  jacobi3d_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, gx, P->b_dev, P->nx, P->ny,
                                                                 P->nz, P->ey, P->ez, P->omega);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_g_bratu2d(const double *x, double *gx, int64_t n, void *stream, void *user) {
  const aa_bratu2d *P = (const aa_bratu2d *)user;
  if (!P || !x || !gx || n != P->s * P->s) return AA_EINVAL;
  bratu2d_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, gx, P->src_dev, P->s,
                                                                P->lambda);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}
