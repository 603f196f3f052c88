// aa_mlp.cu -- kernels of the learned warm start: a multilayer perceptron
// that maps problem parameters to an initial guess x_0, trained on the GPU.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T with BF16 inputs and FP32
// accumulation on the tensor cores (mma.sync m16n8k16), operands staged in
// shared memory with cp.async double buffering and read with ldmatrix, and a
// fused epilogue (bias, GELU, BF16 or FP32 store).  Every product the MLP
// needs is written in this one form: the forward pass directly; the data and
// weight gradients after explicit transposes.
// Elementwise kernels: transpose, GELU derivative, mean-squared-error
// gradient, Adam with FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/aa.h"

namespace {

constexpr int BMt = 128, BNt = 128, BKt = 32;  // block tile
constexpr int GEMM_THREADS = 256;              // 8 warps: 2 (M) x 4 (N), warp tile 64 x 32
constexpr int SPAD = 8;                        // smem row padding (bf16) against bank conflicts
constexpr int SROW = BKt + SPAD;               // 40 bf16 = 80 bytes per smem row

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
  const int n = pred ? 16 : 0;  // zero-fill when out of range
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(smem)), "l"(gmem),
               "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t (&r)[2], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// Loads a BMt x BKt tile of a row-major [rows x K] bf16 matrix (K contiguous)
// into shared memory rows of SROW; requires K % 8 == 0 and 16-byte aligned rows.
__device__ __forceinline__ void load_tile(__nv_bfloat16 *s, const __nv_bfloat16 *g, int ld,
                                          int rows, int K, int r0, int k0) {
  // 128 rows x 32 cols = 512 chunks of 8 bf16; 256 threads x 2
  for (int c = threadIdx.x; c < BMt * (BKt / 8); c += GEMM_THREADS) {
    const int r = c / (BKt / 8), kc = (c % (BKt / 8)) * 8;
    const int gr = r0 + r, gk = k0 + kc;
    const bool ok = gr < rows && gk < K;
    const __nv_bfloat16 *src = ok ? g + (size_t)gr * ld + gk : g;
    cp_async16(s + r * SROW + kc, src, ok);
  }
}

// epi: bit 0 add bias, bit 1 GELU, bit 2 store bf16 (else fp32), bit 3 also
// store the pre-activation (fp32) to P, bit 4 add the product to the fp32 C
// already in place (C += A B^T).
__global__ void __launch_bounds__(GEMM_THREADS)
    gemm_nt_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
                   const __nv_bfloat16 *__restrict__ B, int ldb, void *C, int ldc,
                   const float *__restrict__ bias, float *P, int ldp, int epi) {
  __shared__ __align__(128) __nv_bfloat16 sA[2][BMt * SROW];
  __shared__ __align__(128) __nv_bfloat16 sB[2][BNt * SROW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps
  const int m0 = blockIdx.y * BMt, n0 = blockIdx.x * BNt;
  float acc[4][4][4];  // warp tile 64 x 32: 4 (m16) x 4 (n8)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  const int nk = (K + BKt - 1) / BKt;
  load_tile(sA[0], A, lda, M, K, m0, 0);
  load_tile(sB[0], B, ldb, N, K, n0, 0);
  cp_async_commit();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    cp_async_wait_all();
    __syncthreads();
    if (kt + 1 < nk) {
      load_tile(sA[cur ^ 1], A, lda, M, K, m0, (kt + 1) * BKt);
      load_tile(sB[cur ^ 1], B, ldb, N, K, n0, (kt + 1) * BKt);
      cp_async_commit();
    }
#pragma unroll
    for (int kk = 0; kk < BKt; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = wm * 64 + i * 16 + (lane & 15);
        const int col = kk + (lane >> 4) * 8;
        ldmatrix_x4(af[i], &sA[cur][row * SROW + col]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int row = wn * 32 + j * 8 + (lane & 7);
        const int col = kk + ((lane >> 3) & 1) * 8;
        ldmatrix_x2(bf[j], &sB[cur][row * SROW + col]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  // epilogue
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm * 64 + i * 16 + g + h * 8;
        const int col = n0 + wn * 32 + j * 8 + t4 * 2;
        if (row >= M) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int cc = col + q;
          if (cc >= N) continue;
          float v = acc[i][j][h * 2 + q];
          if (epi & 1) v += bias[cc];
          if (epi & 16) v += ((const float *)C)[(size_t)row * ldc + cc];
          if (epi & 8) P[(size_t)row * ldp + cc] = v;
          if (epi & 2) v = gelu(v);
          if (epi & 4)
            ((__nv_bfloat16 *)C)[(size_t)row * ldc + cc] = __float2bfloat16_rn(v);
          else
            ((float *)C)[(size_t)row * ldc + cc] = v;
        }
      }
}

__global__ void transpose_bf16_kernel(int rows, int cols, const __nv_bfloat16 *__restrict__ in,
                                      int ldi, __nv_bfloat16 *__restrict__ out, int ldo) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[y][threadIdx.x] = in[(size_t)r * ldi + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(size_t)c * ldo + r] = t[threadIdx.x][y];
  }
}

// grad (bf16, in/out) *= GELU'(pre)
__global__ void gelu_bwd_kernel(int64_t n, const float *__restrict__ pre, __nv_bfloat16 *grad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    grad[i] = __float2bfloat16_rn(__bfloat162float(grad[i]) * gelu_grad(pre[i]));
}

// MSE: loss = mean((y - t)^2); dy = 2 (y - t) / count (bf16); partial losses
// per block summed in fixed order by the host.
__global__ void mse_kernel(int64_t n, const float *__restrict__ y, const float *__restrict__ t,
                           float scale, __nv_bfloat16 *dy, double *block_loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * (double)d;
    dy[i] = __float2bfloat16_rn(2.0f * d * scale);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_loss[blockIdx.x] = red[0];
}

// column sums of a [rows x cols] bf16 matrix into fp32 (bias gradient)
__global__ void colsum_kernel(int rows, int cols, const __nv_bfloat16 *__restrict__ g, int ld,
                              float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(g[(size_t)r * ld + c]);
  out[c] = s;
}

__global__ void adam_kernel(int64_t n, float *w, __nv_bfloat16 *wb, const float *__restrict__ g,
                            float *m, float *v, float lr, float b1, float b2, float eps, float c1,
                            float c2, float wd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] + wd * w[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

// Momentum SGD with FP32 master weights, refreshing a split BF16 copy
// w ~ hi + lo (both BF16: about 16 significant bits together).
__global__ void sgd_kernel(int64_t n, float *w, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                           const float *__restrict__ g, float *mom, float lr, float mu, float wd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float mi = mu * mom[i] + g[i] + wd * w[i];
    mom[i] = mi;
    const float wi = w[i] - lr * mi;
    w[i] = wi;
    if (hi) {
      const __nv_bfloat16 h = __float2bfloat16_rn(wi);
      hi[i] = h;
      if (lo) lo[i] = __float2bfloat16_rn(wi - __bfloat162float(h));
    }
  }
}

__global__ void split_bf16_kernel(int64_t n, const float *__restrict__ x, __nv_bfloat16 *hi,
                                  __nv_bfloat16 *lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(x[i] - __bfloat162float(h));
  }
}

__global__ void f32_to_bf16_kernel(int64_t n, const float *__restrict__ x, __nv_bfloat16 *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

int grid1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" int aa_gemm_bf16_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb,
                               void *C, int ldc, const float *bias, float *pre, int ldp, int epi,
                               void *stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return AA_EINVAL;
  if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K || !al16(A) || !al16(B)) return AA_EINVAL;
  if (((epi & 1) && !bias) || ((epi & 8) && !pre)) return AA_EINVAL;
  if ((epi & 16) && (epi & 4)) return AA_EINVAL;  // accumulation is into fp32 C only
  dim3 grid((N + BNt - 1) / BNt, (M + BMt - 1) / BMt);
  if (grid.y > 65535) return AA_EINVAL;
  gemm_nt_kernel<<<grid, GEMM_THREADS, 0, (cudaStream_t)stream>>>(
      M, N, K, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc, bias, pre, ldp,
      epi);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_transpose_bf16(int rows, int cols, const void *in, int ldi, void *out, int ldo,
                                 void *stream) {
  if (rows < 1 || cols < 1 || !in || !out) return AA_EINVAL;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  if (grid.y > 65535) return AA_EINVAL;
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, (cudaStream_t)stream>>>(
      rows, cols, (const __nv_bfloat16 *)in, ldi, (__nv_bfloat16 *)out, ldo);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_gelu_bwd(int64_t n, const float *pre, void *grad, void *stream) {
  if (n < 1 || !pre || !grad) return AA_EINVAL;
  gelu_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(n, pre, (__nv_bfloat16 *)grad);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_mse(int64_t n, const float *y, const float *t, float scale, void *dy,
                      double *block_loss, int nblocks, void *stream) {
  if (n < 1 || !y || !t || !dy || !block_loss || nblocks < 1) return AA_EINVAL;
  mse_kernel<<<nblocks, 256, 0, (cudaStream_t)stream>>>(n, y, t, scale, (__nv_bfloat16 *)dy,
                                                        block_loss);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_colsum_bf16(int rows, int cols, const void *g, int ld, float *out,
                              void *stream) {
  if (rows < 1 || cols < 1 || !g || !out) return AA_EINVAL;
  colsum_kernel<<<(cols + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      rows, cols, (const __nv_bfloat16 *)g, ld, out);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_adam(int64_t n, float *w, void *w_bf16, const float *g, float *m, float *v,
                       float lr, float beta1, float beta2, float eps, int step, float weight_decay,
                       void *stream) {
  if (n < 1 || !w || !g || !m || !v || step < 1) return AA_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(
      n, w, (__nv_bfloat16 *)w_bf16, g, m, v, lr, beta1, beta2, eps, c1, c2, weight_decay);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_f32_to_bf16(int64_t n, const float *x, void *y, void *stream) {
  if (n < 1 || !x || !y) return AA_EINVAL;
  f32_to_bf16_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(n, x, (__nv_bfloat16 *)y);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_sgd(int64_t n, float *w, void *w_hi, void *w_lo, const float *g, float *mom,
                      float lr, float momentum, float weight_decay, void *stream) {
  if (n < 1 || !w || !g || !mom || (w_lo && !w_hi)) return AA_EINVAL;
  sgd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(
      n, w, (__nv_bfloat16 *)w_hi, (__nv_bfloat16 *)w_lo, g, mom, lr, momentum, weight_decay);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}

extern "C" int aa_f32_split_bf16(int64_t n, const float *x, void *hi, void *lo, void *stream) {
  if (n < 1 || !x || !hi || !lo) return AA_EINVAL;
  split_bf16_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(n, x, (__nv_bfloat16 *)hi,
                                                                 (__nv_bfloat16 *)lo);
  return cudaGetLastError() == cudaSuccess ? AA_OK : AA_ECUDA;
}
