// Residual (FuncEval) and Jacobian (JacEval) assembly.
//
// Atomic-free, deterministic two-phase scheme:
//   1. one element kernel computes every tet's contribution into an element
//      buffer (Fe: 4 x 7 rows per tet; Ke: 4 x 4 blocks of 7 x 7 per tet);
//   2. one gather kernel sums, for every node row (resp. BSR block), the buffer
//      slots listed for it in increasing tet order.
// Element rows are routed to node rows by the node flags (strong interface
// coupling, Sec. 2.2): continuity -> p row; fluid momentum -> u rows of
// fluid-only nodes and d rows of interface nodes; mesh motion -> d rows of
// fluid-only nodes; wall momentum -> d rows. Constrained rows receive zeros
// and are written afterwards by the constraint kernels.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "setup.h"

namespace fsi {

namespace {

__device__ __forceinline__ void load_tet(const MeshDev& m, int64_t t, int n[4], uint32_t f[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    n[a] = m.tets[4 * t + a];
    f[a] = m.nflag[n[a]];
  }
}

// reference coordinates relative to vertex 0 (translation-invariant element
// routines; keeps full relative precision of the edges in FP32)
template <class T>
__device__ __forceinline__ void load_X(const MeshDev& m, const int n[4], T Xl[4][3]) {
  const double x0 = m.X[3 * (int64_t)n[0]], y0 = m.X[3 * (int64_t)n[0] + 1], z0 = m.X[3 * (int64_t)n[0] + 2];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Xl[a][0] = T(m.X[3 * (int64_t)n[a]] - x0);
    Xl[a][1] = T(m.X[3 * (int64_t)n[a] + 1] - y0);
    Xl[a][2] = T(m.X[3 * (int64_t)n[a] + 2] - z0);
  }
}

__global__ void k_elem_residual(MeshDev m, MatConst mc, const double* __restrict__ y,
                                const double* __restrict__ y1, const double* __restrict__ y2,
                                double* __restrict__ Fe) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m.T; t += (int64_t)gridDim.x * blockDim.x) {
    int n[4];
    uint32_t f[4];
    load_tet(m, t, n, f);
    double Xl[4][3];
    load_X<double>(m, n, Xl);
    double out[4][7];
    if (t < m.Tf) {
      double u[4][3], p[4], d[4][3], u1[4][3], d1[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double* ya = y + 7 * (int64_t)n[a];
        const double* y1a = y1 + 7 * (int64_t)n[a];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          u[a][i] = ya[i];
          d[a][i] = ya[4 + i];
          u1[a][i] = y1a[i];
          d1[a][i] = y1a[4 + i];
        }
        p[a] = ya[3];
      }
      double Rm[4][3], Rc[4], Rh[4][3];
      fluid_element<double, double>(Xl, u, p, d, u1, d1, mc, Rm, Rc, Rh);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const bool uc = f[a] & NF_U_CONSTR, pc = f[a] & NF_P_IDENT, dz = f[a] & NF_D_ZERO, itf = f[a] & NF_ITF;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          out[a][i] = uc ? 0.0 : Rm[a][i];
          out[a][4 + i] = dz ? 0.0 : (itf ? Rm[a][i] : Rh[a][i]);
        }
        out[a][3] = pc ? 0.0 : Rc[a];
      }
    } else {
      double d[4][3], d1[4][3], d2[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          d[a][i] = y[7 * (int64_t)n[a] + 4 + i];
          d1[a][i] = y1[7 * (int64_t)n[a] + 4 + i];
          d2[a][i] = y2[7 * (int64_t)n[a] + 4 + i];
        }
      double Rw[4][3];
      wall_element<double, double>(Xl, d, d1, d2, mc, Rw);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const bool dz = f[a] & NF_D_ZERO;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          out[a][i] = 0.0;
          out[a][4 + i] = dz ? 0.0 : Rw[a][i];
        }
        out[a][3] = 0.0;
      }
    }
    double* o = Fe + 28 * t;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int r = 0; r < 7; ++r) o[7 * a + r] = out[a][r];
  }
}

__global__ void k_gather_residual(int64_t N, const int64_t* __restrict__ nptr, const int32_t* __restrict__ nsrc,
                                  const double* __restrict__ Fe, double* __restrict__ F) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 7 * N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / 7;
    const int r = (int)(idx - 7 * i);
    double s = 0.0;
    for (int64_t c = nptr[i]; c < nptr[i + 1]; ++c) s += Fe[7 * (int64_t)nsrc[c] + r];
    F[idx] = s;
  }
}

__global__ void k_constraint_residual(MeshDev m, MatConst mc, double t, const double* __restrict__ y,
                                      const double* __restrict__ y1, double* __restrict__ F) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t f = m.nflag[i];
    const double* yi = y + 7 * i;
    double* Fi = F + 7 * i;
    if (f & NF_U_KIN) {
      const double* y1i = y1 + 7 * i;
      const double idt = 1.0 / mc.dt;
      for (int c = 0; c < 3; ++c) Fi[c] = yi[c] - (yi[4 + c] - y1i[4 + c]) * idt;
    }
    if (f & NF_U_IDENT)
      for (int c = 0; c < 3; ++c) Fi[c] = yi[c];
    if (f & NF_P_IDENT) Fi[3] = yi[3];
    if (f & NF_D_ZERO)
      for (int c = 0; c < 3; ++c) Fi[4 + c] = yi[4 + c];
    if (f & NF_U_INLET) {
      const double* in = m.inlet + INLET_STRIDE * m.nprob[i];
      const double rx = m.X[3 * i] - in[0], ry = m.X[3 * i + 1] - in[1], rz = m.X[3 * i + 2] - in[2];
      const double ax = rx * in[3] + ry * in[4] + rz * in[5];
      const double r2 = (rx * rx + ry * ry + rz * rz) - ax * ax;
      const double U = in[7] * (1.0 + in[8] * sin(2.0 * 3.141592653589793 * in[9] * t + in[10]));
      const double prof = fmax(0.0, 1.0 - r2 / (in[6] * in[6]));
      for (int c = 0; c < 3; ++c) Fi[c] = yi[c] - U * prof * in[3 + c];
    }
  }
}

// One Jacobian column per thread: 28 threads per tet (column = node b, dof k),
// forward-mode derivative of the element residual along that column. Inputs
// are already in the arithmetic type T: per-tet reference coordinates relative
// to vertex 0 (Xl, 12 per tet) and node states (y, y_old, y_older), so the FP32
// kernel runs no FP64 instruction.
constexpr int JAC_TETS_PER_BLOCK = 8;

template <class T>
__global__ void __launch_bounds__(28 * JAC_TETS_PER_BLOCK)
k_elem_jacobian(MeshDev m, MatConst mc, const T* __restrict__ Xl, const T* __restrict__ y,
                const T* __restrict__ y1, const T* __restrict__ y2, T* __restrict__ Ke, int64_t t0, int64_t t1) {
  const int tl = threadIdx.x / 28;
  const int colid = threadIdx.x - 28 * tl;
  const int b = colid / 7, k = colid - 7 * (colid / 7);
  for (int64_t t = t0 + blockIdx.x * (int64_t)JAC_TETS_PER_BLOCK + tl; t < t1;
       t += (int64_t)gridDim.x * JAC_TETS_PER_BLOCK) {
    int n[4];
    uint32_t f[4];
    load_tet(m, t, n, f);
    T X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) X[a][i] = Xl[12 * t + 3 * a + i];
    T out[4][7];
    if (t < m.Tf) {
      Dual<T> u[4][3], p[4], d[4][3];
      T u1[4][3], d1[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T* ya = y + 7 * (int64_t)n[a];
        const T* y1a = y1 + 7 * (int64_t)n[a];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          u[a][i] = Dual<T>(ya[i], (a == b && k == i) ? T(1) : T(0));
          d[a][i] = Dual<T>(ya[4 + i], (a == b && k == 4 + i) ? T(1) : T(0));
          u1[a][i] = y1a[i];
          d1[a][i] = y1a[4 + i];
        }
        p[a] = Dual<T>(ya[3], (a == b && k == 3) ? T(1) : T(0));
      }
      Dual<T> Rm[4][3], Rc[4], Rh[4][3];
      fluid_element<Dual<T>, T>(X, u, p, d, u1, d1, mc, Rm, Rc, Rh);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const bool uc = f[a] & NF_U_CONSTR, pc = f[a] & NF_P_IDENT, dz = f[a] & NF_D_ZERO, itf = f[a] & NF_ITF;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          out[a][i] = uc ? T(0) : Rm[a][i].d;
          out[a][4 + i] = dz ? T(0) : (itf ? Rm[a][i].d : Rh[a][i].d);
        }
        out[a][3] = pc ? T(0) : Rc[a].d;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int r = 0; r < 7; ++r) out[a][r] = T(0);
      if (k >= 4) {
        Dual<T> d[4][3];
        T d1[4][3], d2[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            d[a][i] = Dual<T>(y[7 * (int64_t)n[a] + 4 + i], (a == b && k == 4 + i) ? T(1) : T(0));
            d1[a][i] = y1[7 * (int64_t)n[a] + 4 + i];
            d2[a][i] = y2[7 * (int64_t)n[a] + 4 + i];
          }
        Dual<T> Rw[4][3];
        wall_element<Dual<T>, T>(X, d, d1, d2, mc, Rw);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const bool dz = f[a] & NF_D_ZERO;
#pragma unroll
          for (int i = 0; i < 3; ++i) out[a][4 + i] = dz ? T(0) : Rw[a][i].d;
        }
      }
    }
    // Ke[t - t0][a][b][r][k]
    T* o = Ke + 784 * (t - t0) + 49 * b + k;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int r = 0; r < 7; ++r) o[196 * a + 7 * r] = out[a][r];
  }
}

__global__ void k_states_to_float(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                  const double* __restrict__ c, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = (float)a[i];
    out[n + i] = (float)b[i];
    out[2 * n + i] = (float)c[i];
  }
}

// Sum into each block the element blocks of the tets [t0, t1) (the buffer holds
// those tets only). Each block's contributions are listed in increasing tet
// order, so a chunk of tets is a contiguous part of every list; the first chunk
// starts the sum at zero, the next ones continue it from vals, so the additions
// happen in the same order as in a single pass (bitwise the same result).
template <class T>
__global__ void k_gather_jacobian(int64_t nnzb, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bsrc,
                                  const T* __restrict__ Ke, T* __restrict__ vals, int64_t t0, int64_t t1) {
  const int64_t lo = 16 * t0, hi = 16 * t1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 49 * nnzb;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kb = idx / 49;
    const int e = (int)(idx - 49 * kb);
    T s = t0 == 0 ? T(0) : vals[idx];
    for (int64_t c = bptr[kb]; c < bptr[kb + 1]; ++c) {
      const int64_t src = bsrc[c];
      if (src < lo) continue;
      if (src >= hi) break;
      s += Ke[49 * (src - lo) + e];
    }
    vals[idx] = s;
  }
}

template <class T>
__global__ void k_constraint_jacobian(MeshDev m, MatConst mc, const int32_t* __restrict__ diag, T* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t f = m.nflag[i];
    T* D = vals + 49 * (int64_t)diag[i];
    if (f & (NF_U_KIN | NF_U_IDENT | NF_U_INLET))
      for (int c = 0; c < 3; ++c) D[8 * c] = T(1);
    if (f & NF_U_KIN)
      for (int c = 0; c < 3; ++c) D[7 * c + 4 + c] = T(-1.0 / mc.dt);
    if (f & NF_P_IDENT) D[8 * 3] = T(1);
    if (f & NF_D_ZERO)
      for (int c = 4; c < 7; ++c) D[8 * c] = T(1);
  }
}

inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = 152 * 64;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void launch_elem_residual(const MeshDev& m, const MatConst& mc, const double* y, const double* y1,
                          const double* y2, double* Fe, cudaStream_t s) {
  if (m.T == 0) return;
  k_elem_residual<<<grid_for(m.T, 128), 128, 0, s>>>(m, mc, y, y1, y2, Fe);
}

void launch_gather_residual(const MeshDev& m, const int64_t* nptr, const int32_t* nsrc, const double* Fe,
                            double* F, cudaStream_t s) {
  k_gather_residual<<<grid_for(7 * m.N, 256), 256, 0, s>>>(m.N, nptr, nsrc, Fe, F);
}

void launch_constraint_residual(const MeshDev& m, const MatConst& mc, double t, const double* y,
                                const double* y1, double* F, cudaStream_t s) {
  k_constraint_residual<<<grid_for(m.N, 256), 256, 0, s>>>(m, mc, t, y, y1, F);
}

template <class T>
void launch_elem_jacobian(const MeshDev& m, const MatConst& mc, const T* Xl, const T* y, const T* y1, const T* y2,
                          T* Ke, int64_t t0, int64_t t1, cudaStream_t s) {
  if (t1 <= t0) return;
  int64_t blocks = (t1 - t0 + JAC_TETS_PER_BLOCK - 1) / JAC_TETS_PER_BLOCK;
  if (blocks > 152 * 256) blocks = 152 * 256;
  k_elem_jacobian<T><<<(int)blocks, 28 * JAC_TETS_PER_BLOCK, 0, s>>>(m, mc, Xl, y, y1, y2, Ke, t0, t1);
}

void launch_states_to_float(int64_t n, const double* a, const double* b, const double* c, float* out,
                            cudaStream_t s) {
  k_states_to_float<<<grid_for(n, 256), 256, 0, s>>>(n, a, b, c, out);
}

template <class T>
void launch_gather_jacobian(int64_t nnzb, const int64_t* bptr, const int32_t* bsrc, const T* Ke, T* vals,
                            int64_t t0, int64_t t1, cudaStream_t s) {
  k_gather_jacobian<T><<<grid_for(49 * nnzb, 256), 256, 0, s>>>(nnzb, bptr, bsrc, Ke, vals, t0, t1);
}

template <class T>
void launch_constraint_jacobian(const MeshDev& m, const MatConst& mc, const int32_t* diag, T* vals,
                                cudaStream_t s) {
  k_constraint_jacobian<T><<<grid_for(m.N, 256), 256, 0, s>>>(m, mc, diag, vals);
}

template void launch_elem_jacobian<double>(const MeshDev&, const MatConst&, const double*, const double*,
                                           const double*, const double*, double*, int64_t, int64_t, cudaStream_t);
template void launch_elem_jacobian<float>(const MeshDev&, const MatConst&, const float*, const float*,
                                          const float*, const float*, float*, int64_t, int64_t, cudaStream_t);
template void launch_gather_jacobian<double>(int64_t, const int64_t*, const int32_t*, const double*, double*,
                                             int64_t, int64_t, cudaStream_t);
template void launch_gather_jacobian<float>(int64_t, const int64_t*, const int32_t*, const float*, float*,
                                            int64_t, int64_t, cudaStream_t);
template void launch_constraint_jacobian<double>(const MeshDev&, const MatConst&, const int32_t*, double*,
                                                 cudaStream_t);
template void launch_constraint_jacobian<float>(const MeshDev&, const MatConst&, const int32_t*, float*,
                                                cudaStream_t);

}  // namespace fsi
