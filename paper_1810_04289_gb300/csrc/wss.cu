// Wall shear stress on the inner wall (the results section of the paper, after
// Eq. 16): on every face shared by a fluid tet and a wall tet,
//   WSS = sigma n - (sigma n . n) n,  sigma = -p I + 2 mu eps(u)   (Eq. 3),
// with eps(u) of the P1 fluid tet on the current configuration x = X + d, p at
// the face centroid and n the unit normal out of the fluid; and per problem the
// spatially averaged WSS, SAWSS = sum |WSS| area / sum area (the surface
// integral of the WSS magnitude normalised by the wall area).
//
// One thread per face writes the face's vector, |WSS| area and area; one block
// per problem then sums its faces in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "element.cuh"
#include "kernels.cuh"

namespace fsi {

namespace {

__global__ void k_wss_faces(MeshDev m, double mu, int64_t nf, const int64_t* __restrict__ face,
                            const double* __restrict__ y, double* __restrict__ wss, double* __restrict__ marea,
                            double* __restrict__ area) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = face[i] >> 2;
    const int f = (int)(face[i] & 3);
    double x[4][3], u[4][3], p[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t v = m.tets[4 * t + a];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        x[a][k] = m.X[3 * v + k] + y[7 * v + 4 + k];
        u[a][k] = y[7 * v + k];
      }
      p[a] = y[7 * v + 3];
    }
    double g[4][3], vol;
    tet_gradients<double>(x, g, vol);
    // eps = sym(grad u), (grad u)_ij = sum_a u_a,i dN_a/dx_j
    double G[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) G[r][c] = u[0][r] * g[0][c] + u[1][r] * g[1][c] + u[2][r] * g[2][c] + u[3][r] * g[3][c];
    // the face: the three vertices other than f
    int fv[3], k3 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (a != f) fv[k3++] = a;
    double e1[3], e2[3], cr[3], ctr[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e1[k] = x[fv[1]][k] - x[fv[0]][k];
      e2[k] = x[fv[2]][k] - x[fv[0]][k];
      ctr[k] = (x[fv[0]][k] + x[fv[1]][k] + x[fv[2]][k]) / 3.0;
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double n[3] = {cr[0] / len, cr[1] / len, cr[2] / len};
    const double side = n[0] * (ctr[0] - x[f][0]) + n[1] * (ctr[1] - x[f][1]) + n[2] * (ctr[2] - x[f][2]);
    if (side < 0) {
      n[0] = -n[0];
      n[1] = -n[1];
      n[2] = -n[2];
    }
    const double pf = (p[fv[0]] + p[fv[1]] + p[fv[2]]) / 3.0;
    double sn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double en = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) en += 0.5 * (G[r][c] + G[c][r]) * n[c];
      sn[r] = -pf * n[r] + 2.0 * mu * en;
    }
    const double snn = sn[0] * n[0] + sn[1] * n[1] + sn[2] * n[2];
    double w2 = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double wr = sn[r] - snn * n[r];
      if (wss) wss[3 * i + r] = wr;
      w2 += wr * wr;
    }
    const double A = 0.5 * len;
    marea[i] = sqrt(w2) * A;
    area[i] = A;
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sawss[p] = sum of marea / sum of area over the faces [fb[p], fb[p+1]) of problem p
__global__ void __launch_bounds__(256) k_wss_reduce(const int64_t* __restrict__ fb, const double* __restrict__ marea,
                                                    const double* __restrict__ area, double* __restrict__ sawss) {
  __shared__ double s_m[8], s_a[8];
  const int p = blockIdx.x;
  double m = 0.0, a = 0.0;
  for (int64_t i = fb[p] + threadIdx.x; i < fb[p + 1]; i += blockDim.x) {
    m += marea[i];
    a += area[i];
  }
  m = wsum(m);
  a = wsum(a);
  if ((threadIdx.x & 31) == 0) {
    s_m[threadIdx.x >> 5] = m;
    s_a[threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, ta = 0.0;
    for (int w = 0; w < 8; ++w) {
      tm += s_m[w];
      ta += s_a[w];
    }
    sawss[p] = ta > 0.0 ? tm / ta : 0.0;
  }
}

}  // namespace

void launch_wss(const MeshDev& m, double mu, int64_t nf, const int64_t* face, const int64_t* fb, int32_t P,
                const double* y, double* wss, double* marea, double* area, double* sawss, cudaStream_t s) {
  if (nf > 0) {
    int64_t g = (nf + 127) / 128;
    if (g > 152 * 16) g = 152 * 16;
    k_wss_faces<<<(int)g, 128, 0, s>>>(m, mu, nf, face, y, wss, marea, area);
  }
  k_wss_reduce<<<P, 256, 0, s>>>(fb, marea, area, sawss);
}

}  // namespace fsi
