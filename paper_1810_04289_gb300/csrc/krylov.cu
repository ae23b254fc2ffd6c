// FP64 vector kernels of the Krylov loop: multi-dot products for classical
// Gram-Schmidt (twice), multi-axpy, norms, scaling, Givens rotations and the
// Hessenberg least-squares solve. Reductions use a fixed grid of RED_BLOCKS
// blocks and a second pass in fixed order, so results are bitwise
// reproducible run to run.
//
// Kernels that run inside a captured GMRES cycle take a guard pointer: while
// *guard == 0 (the cycle has converged or broken down) they return at once, so
// the remaining iterations of the captured cycle cost only their launches.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fsi {

namespace {

constexpr int RB = 256;   // threads per reduction block
constexpr int MD = 8;     // vectors per multi-dot pass

__device__ __forceinline__ bool off(const int* guard) { return guard && *guard == 0; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[blockIdx.x * ldp + k] = sum over this block's rows of V_k . w
__global__ void __launch_bounds__(RB) k_mdot(int64_t n, int32_t nv, const double* __restrict__ V, int64_t ldv,
                                             const double* __restrict__ w, double* __restrict__ partial,
                                             int32_t ldp, const int* guard) {
  if (off(guard)) return;
  __shared__ double red[MD][RB / 32];
  const int k0 = blockIdx.y * MD;
  double acc[MD];
#pragma unroll
  for (int k = 0; k < MD; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < MD; ++k)
      if (k0 + k < nv) acc[k] += V[(int64_t)(k0 + k) * ldv + i] * wi;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < MD; ++k) {
    double v = warp_sum(acc[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < MD && k0 + threadIdx.x < nv) {
    double v = 0.0;
    for (int q = 0; q < RB / 32; ++q) v += red[threadIdx.x][q];
    partial[(int64_t)blockIdx.x * ldp + k0 + threadIdx.x] = v;
  }
}

__global__ void k_reduce_partials(int32_t nv, const double* __restrict__ partial, int32_t ldp, int32_t nb,
                                  double* __restrict__ out, int take_sqrt, const int* guard) {
  if (off(guard)) return;
  __shared__ double red[RB / 32];
  for (int k = 0; k < nv; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[(int64_t)b * ldp + k];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
      out[k] = take_sqrt ? sqrt(s) : s;
    }
    __syncthreads();
  }
}

// w -= sum_k h[k] V_k
__global__ void k_maxpy(int64_t n, int32_t nv, const double* __restrict__ V, int64_t ldv,
                        const double* __restrict__ h, double* __restrict__ w, const int* guard) {
  if (off(guard)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nv; ++k) s -= h[k] * V[(int64_t)k * ldv + i];
    w[i] = s;
  }
}

__global__ void k_norm_partial(int64_t n, const double* __restrict__ x, double* __restrict__ partial,
                               const int* guard) {
  if (off(guard)) return;
  __shared__ double red[RB / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) acc += x[i] * x[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < RB / 32; ++q) s += red[q];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_scale_inv(int64_t n, const double* __restrict__ x, const double* __restrict__ scal,
                            double* __restrict__ y, const int* guard) {
  if (off(guard)) return;
  const double a = *scal;
  const double inv = a != 0.0 ? 1.0 / a : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (b != 0.0 ? b * y[i] : 0.0);
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// Hcol[k] = a[k] + b[k] (the two classical Gram-Schmidt passes)
__global__ void k_add_small(int32_t nv, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ out, const int* guard) {
  if (off(guard)) return;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) out[k] = a[k] + b[k];
}

// start of a cycle: g = beta e_1 (beta = *scal), the cycle is active, no columns yet
__global__ void k_cycle_init(double* __restrict__ g, int32_t ldh, const double* __restrict__ scal,
                             int* __restrict__ active, int* __restrict__ kcols) {
  for (int k = threadIdx.x; k < ldh; k += blockDim.x) g[k] = k == 0 ? *scal : 0.0;
  if (threadIdx.x == 0) {
    *active = 1;
    *kcols = 0;
  }
}

// Givens update of Hessenberg column j (column-major, leading dimension ldh):
// apply the previous rotations, form the one that zeroes H[j+1][j], rotate the
// right-hand side g; |g[j+1]| is the GMRES residual norm. Stops the cycle when
// it reaches *target or the Krylov space is exhausted (H[j+1][j] = 0).
__global__ void k_givens(double* __restrict__ H, int32_t ldh, int32_t j, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res,
                         const double* __restrict__ target, int* __restrict__ active, int* __restrict__ kcols) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (active && *active == 0) return;
  double* h = H + (int64_t)j * ldh;
  const double sub = h[j + 1];
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double r = hypot(a, b);
  double c = 1.0, sv = 0.0;
  if (r > 0.0) {
    c = a / r;
    sv = b / r;
  }
  cs[j] = c;
  sn[j] = sv;
  h[j] = r;
  h[j + 1] = 0.0;
  const double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -sv * gj;
  const double rn = fabs(g[j + 1]);
  *res = rn;
  if (kcols) *kcols = j + 1;
  if (active && target && (!(rn > *target) || sub == 0.0)) *active = 0;
}

// y = R^{-1} g for the k x k upper-triangular rotated Hessenberg R (k = *kdev if given)
__global__ void k_lsq(const double* __restrict__ H, int32_t ldh, int32_t k, const int* __restrict__ kdev,
                      const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (kdev) k = *kdev;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int jj = i + 1; jj < k; ++jj) s -= H[(int64_t)jj * ldh + i] * y[jj];
    const double d = H[(int64_t)i * ldh + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// x += sum_{q < k} y_q Z_q
__global__ void k_update_x(int64_t n, const double* __restrict__ Z, int64_t ldz, const double* __restrict__ y,
                           const int* __restrict__ kdev, double* __restrict__ x) {
  const int k = *kdev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int q = 0; q < k; ++q) s += y[q] * Z[(int64_t)q * ldz + i];
    x[i] = s;
  }
}

inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = 152 * 32;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void launch_mdot(int64_t n, int32_t nv, const double* V, int64_t ldv, const double* w, double* partial,
                 double* out, const int* guard, cudaStream_t s) {
  dim3 grid(RED_BLOCKS, (nv + MD - 1) / MD);
  k_mdot<<<grid, RB, 0, s>>>(n, nv, V, ldv, w, partial, nv, guard);
  k_reduce_partials<<<1, RB, 0, s>>>(nv, partial, nv, RED_BLOCKS, out, 0, guard);
}

void launch_maxpy(int64_t n, int32_t nv, const double* V, int64_t ldv, const double* h, double* w,
                  const int* guard, cudaStream_t s) {
  k_maxpy<<<grid_for(n, 256), 256, 0, s>>>(n, nv, V, ldv, h, w, guard);
}

void launch_norm(int64_t n, const double* x, double* partial, double* out, const int* guard, cudaStream_t s) {
  k_norm_partial<<<RED_BLOCKS, RB, 0, s>>>(n, x, partial, guard);
  k_reduce_partials<<<1, RB, 0, s>>>(1, partial, 1, RED_BLOCKS, out, 1, guard);
}

void launch_scale_inv(int64_t n, const double* x, const double* scal, double* y, const int* guard,
                      cudaStream_t s) {
  k_scale_inv<<<grid_for(n, 256), 256, 0, s>>>(n, x, scal, y, guard);
}

void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  k_axpby<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y, out);
}

void launch_copy(int64_t n, const double* x, double* y, cudaStream_t s) {
  cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

void launch_fill(int64_t n, double v, double* x, cudaStream_t s) {
  k_fill<<<grid_for(n, 256), 256, 0, s>>>(n, v, x);
}

void launch_add_small(int32_t nv, const double* a, const double* b, double* out, const int* guard, cudaStream_t s) {
  k_add_small<<<1, 64, 0, s>>>(nv, a, b, out, guard);
}

void launch_cycle_init(double* g, int32_t ldh, const double* scal, int* active, int* kcols, cudaStream_t s) {
  k_cycle_init<<<1, 64, 0, s>>>(g, ldh, scal, active, kcols);
}

void launch_givens(double* H, int32_t ldh, int32_t j, double* cs, double* sn, double* g, double* res,
                   const double* target, int* active, int* kcols, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, g, res, target, active, kcols);
}

void launch_lsq(const double* H, int32_t ldh, int32_t k, const int* kdev, const double* g, double* y,
                cudaStream_t s) {
  k_lsq<<<1, 32, 0, s>>>(H, ldh, k, kdev, g, y);
}

void launch_update_x(int64_t n, const double* Z, int64_t ldz, const double* y, const int* kdev, double* x,
                     cudaStream_t s) {
  k_update_x<<<grid_for(n, 256), 256, 0, s>>>(n, Z, ldz, y, kdev, x);
}

}  // namespace fsi
