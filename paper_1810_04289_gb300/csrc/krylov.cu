// FP64 vector kernels of the batched Krylov loop. The unknowns of P independent
// problems are stored one after the other; every reduction is segmented by
// problem: a fixed table of chunks (each inside one problem) is reduced by one
// block per chunk, and the last block of a problem to finish (a per-problem
// counter) sums that problem's chunk partials in fixed order, so results are
// bitwise reproducible run to run, independent problems never mix, and a
// reduction is one launch per group width (a multi-dot: one for its full groups
// of 8 vectors, one for a partial last group).
// Per-problem Arnoldi scalars: H (column-major (m+1) x m per problem), g, Givens
// cs/sn, residual estimates, stop flags.
//
// Kernels that run inside a captured GMRES cycle take a guard pointer: while
// *guard == 0 (every problem has converged or broken down) they return at once,
// so the rest of the captured cycle costs only its launches.
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

// out[p * ldo + k] = sum over the dofs of problem p of V_k . w (V null: w . w,
// and take_sqrt gives the 2-norm). Block (c, y) forms the partials of chunk c
// for the vectors of group g = g0 + y, 8g .. 8g + W - 1 (those below nv); the
// last block of problem p for group g sums the problem's partials (one warp per
// vector, lanes over the chunks in fixed order) and resets the counter.
// With nself = 1 there is one more output, index nv_v = nv - 1: w . w itself.
// Each thread takes U elements per trip (loads in flight); the kernel is bound by
// the FP64 pipe (one FMA per loaded operand) or, for narrow groups, by latency,
// so the full groups run with W = 8, U = 2 and a partial last group in its own
// launch with a narrower W and a deeper U (fewer registers, more loads in flight).
template <int W, int U>
__global__ void __launch_bounds__(RB) k_seg_mdot(SegDev sg, int32_t nv, int32_t g0, const double* __restrict__ V,
                                                 int64_t ldv, const double* __restrict__ w,
                                                 double* __restrict__ partial, double* __restrict__ out,
                                                 int32_t ldo, int take_sqrt, int nself, const int* guard) {
  if (off(guard)) return;
  __shared__ double red[W][RB / 32];
  __shared__ int s_last;
  const int c = blockIdx.x;
  const int g = g0 + blockIdx.y;
  const int k0 = g * MD;
  const int64_t i0 = sg.chunk_beg[c], i1 = sg.chunk_beg[c + 1];
  double acc[W];
#pragma unroll
  for (int k = 0; k < W; ++k) acc[k] = 0.0;
  const int nvv = nv - nself;  // vectors of V; the rest is w itself
  // vector k of this group: V_{k0+k} while k0 + k < nvv, else w (the self product)
  const double* src[W];
#pragma unroll
  for (int k = 0; k < W; ++k) src[k] = (V && k0 + k < nvv) ? V + (int64_t)(k0 + k) * ldv : w;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += U * RB) {
    double wv[U], v[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iu = i + u * RB;
      const bool in = iu < i1;
      wv[u] = in ? w[iu] : 0.0;
#pragma unroll
      for (int k = 0; k < W; ++k) v[u][k] = (k0 + k < nv && in) ? src[k][iu] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (k0 + k < nv) acc[k] += v[u][k] * wv[u];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    if (k0 + k < nv) {
      const double v = warp_sum(acc[k]);
      if (lane == 0) red[k][warp] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < W && k0 + threadIdx.x < nv) {
    double v = 0.0;
    for (int q = 0; q < RB / 32; ++q) v += red[threadIdx.x][q];
    partial[(int64_t)c * nv + k0 + threadIdx.x] = v;
  }
  // publish the partials, then count this block in
  __threadfence();
  __syncthreads();
  const int p = sg.node_prob[i0 / 7];
  const int64_t c0 = sg.prob_chunk[p], c1 = sg.prob_chunk[p + 1];
  int* cnt = sg.counter + (int64_t)p * SEG_GROUPS + g;
  if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1) == (int)(c1 - c0) - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int k = k0 + warp;
  if (warp < W && k < nv) {
    double v = 0.0;
    for (int64_t cc = c0 + lane; cc < c1; cc += 32) v += __ldcg(partial + cc * nv + k);
    v = warp_sum(v);
    if (lane == 0) out[(int64_t)p * ldo + k] = take_sqrt ? sqrt(v) : v;
  }
  if (threadIdx.x == 0) *cnt = 0;
}

// w_i -= sum_k h[p(i)][k] V_k[i], then (scal non-null) w_i *= scal[p(i)]
__global__ void k_seg_maxpy(SegDev sg, int64_t n, int32_t nv, const double* __restrict__ V, int64_t ldv,
                            const double* __restrict__ h, int32_t ldh, double* __restrict__ w,
                            const double* __restrict__ scal, const int* guard) {
  if (off(guard)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = sg.node_prob[i / 7];
    const double* hp = h + (int64_t)p * ldh;
    double s = w[i];
    for (int k = 0; k < nv; ++k) s -= hp[k] * V[(int64_t)k * ldv + i];
    w[i] = scal ? s * scal[p] : s;
  }
}

// y_i = x_i / scal[p(i) * lds] (0 where the scale is 0). The reciprocal is
// formed once per problem a thread meets (consecutive elements of a thread
// mostly share their problem), not once per element: y_i = x_i * (1 / a).
__global__ void k_seg_scale_inv(SegDev sg, int64_t n, const double* __restrict__ x, const double* __restrict__ scal,
                                int32_t lds, double* __restrict__ y, const int* guard) {
  if (off(guard)) return;
  int pc = -1;
  double inv = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = sg.node_prob[i / 7];
    if (p != pc) {
      const double a = scal[(int64_t)p * lds];
      inv = a != 0.0 ? 1.0 / a : 0.0;
      pc = p;
    }
    y[i] = x[i] * inv;
  }
}

// Classical Gram-Schmidt twice with the new vector's norm taken from the second
// pass: after w1 = w0 - V h1 the second pass's dots h2 = V^T w1 come with
// ||w1||^2 (k_seg_mdot with the self product), and since V is orthonormal,
// ||w1 - V h2||^2 = ||w1||^2 - ||h2||^2. The second update then scales in the
// same sweep (k_seg_maxpy with scal), so the step needs no norm or scaling sweep.
//
// For every problem p, hb[p][0..j] = h2 and hb[p][j+1] = ||w1||^2: where
// ||w1||^2 - ||h2||^2 keeps at least 3/4 of ||w1||^2 (the subtraction then loses
// under two bits) H[p][j+1][j] (hsub + p * ldsub) is its square root and inv[p]
// the reciprocal (0 for a zero norm); elsewhere (only as a Krylov space is
// exhausted; for every problem with force = 1, tests of that path) inv[p] = 1,
// unsafe[p] = 1 and *flag = 1: the norm is then formed from the updated vector
// by the guarded k_seg_norm_fix path.
__global__ void k_seg_norm_pythagoras(int32_t P, const double* __restrict__ hb, int32_t lda, int32_t j,
                                      double* __restrict__ hsub, int64_t ldsub, double* __restrict__ inv,
                                      int* __restrict__ unsafe, int* __restrict__ flag, int force,
                                      const int* guard) {
  __shared__ int s_any;
  if (off(guard)) {
    if (threadIdx.x == 0) *flag = 0;
    return;
  }
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const double* h = hb + (int64_t)p * lda;
    const double s = h[j + 1];
    double q = 0.0;
    for (int k = 0; k <= j; ++k) q += h[k] * h[k];
    const double b2 = s - q;
    if (!force && b2 >= 0.75 * s) {
      const double b = sqrt(b2);
      hsub[(int64_t)p * ldsub] = b;
      inv[p] = b > 0.0 ? 1.0 / b : 0.0;
      unsafe[p] = 0;
    } else {
      inv[p] = 1.0;
      unsafe[p] = 1;
      atomicOr(&s_any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *flag = s_any;
}

// the fallback of k_seg_norm_pythagoras, after nrm[p] = ||w_p|| of the updated
// vector: H[p][j+1][j] = nrm[p] and scal[p] = nrm[p] where unsafe[p], scal[p] = 1
// elsewhere (the vector is then divided by scal)
__global__ void k_seg_norm_fix(int32_t P, const double* __restrict__ nrm, const int* __restrict__ unsafe,
                               double* __restrict__ hsub, int64_t ldsub, double* __restrict__ scal,
                               const int* guard) {
  if (off(guard)) return;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    if (unsafe[p]) {
      hsub[(int64_t)p * ldsub] = nrm[p];
      scal[p] = nrm[p];
    } else {
      scal[p] = 1.0;
    }
  }
}

// start of a cycle for every problem: g = beta e_1, active while beta > target
__global__ void k_seg_cycle_init(int32_t P, double* __restrict__ g, int32_t ldg, const double* __restrict__ beta,
                                 const double* __restrict__ target, int* __restrict__ active, int* __restrict__ kcols,
                                 int* __restrict__ any) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    for (int k = 0; k < ldg; ++k) g[(int64_t)p * ldg + k] = k == 0 ? beta[p] : 0.0;
    const int a = beta[p] > target[p] ? 1 : 0;
    active[p] = a;
    kcols[p] = 0;
    if (a) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *any = s_any;
}

// Selective reorthogonalisation (the criterion of Daniel, Gragg, Kaufman and
// Stewart, 1976): after one classical Gram-Schmidt pass, a second pass is needed
// where the pass removed more than 1 - 1/sqrt(2) of the vector's norm, i.e.
// where ||w_after||^2 < ||w_before||^2 / 2. For every active problem p: s0 =
// ||w_before||^2 (ws[p * lda]), t = ||w_after|| (nrm[p * ldn]); the second-pass
// coefficients hb[p][0..j] are zeroed (a second pass, if it runs, overwrites
// them); *flag = some active problem needs the second pass.
__global__ void k_seg_reorth_decide(int32_t P, const double* __restrict__ ws, const double* __restrict__ nrm,
                                    int32_t ldn, double* __restrict__ hb, int32_t lda, int32_t j,
                                    const int* __restrict__ active, int* __restrict__ flag) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    for (int i = 0; i <= j; ++i) hb[(int64_t)p * lda + i] = 0.0;
    const double s0 = ws[(int64_t)p * lda], t = nrm[(int64_t)p * ldn];
    if (active[p] && t * t < 0.5 * s0) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *flag = s_any;
}

// Givens update of column j of every active problem's Hessenberg (formed here
// as the sum of the two Gram-Schmidt passes; H[j+1][j] is already in place): apply the
// previous rotations, form the one that zeroes H[j+1][j], rotate g; |g[j+1]|
// is that problem's GMRES residual. A problem stops at its target or when its
// Krylov space is exhausted (H[j+1][j] = 0). *any = some problem still active.
__global__ void k_seg_givens(int32_t P, const double* __restrict__ ha, const double* __restrict__ hb, int32_t lda,
                             double* __restrict__ H, int32_t ldh, int32_t m, int32_t j,
                             double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                             double* __restrict__ res, const double* __restrict__ target, int* __restrict__ active,
                             int* __restrict__ kcols, int* __restrict__ any) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    if (active[p]) {
      double* h = H + (int64_t)p * ldh * m + (int64_t)j * ldh;
      for (int i = 0; i <= j; ++i) h[i] = ha[(int64_t)p * lda + i] + hb[(int64_t)p * lda + i];
      double* c_ = cs + (int64_t)p * m;
      double* s_ = sn + (int64_t)p * m;
      double* gp = g + (int64_t)p * ldh;
      const double sub = h[j + 1];
      for (int i = 0; i < j; ++i) {
        const double a = h[i], b = h[i + 1];
        h[i] = c_[i] * a + s_[i] * b;
        h[i + 1] = -s_[i] * a + c_[i] * b;
      }
      const double a = h[j], b = h[j + 1];
      const double r = hypot(a, b);
      double c = 1.0, sv = 0.0;
      if (r > 0.0) {
        c = a / r;
        sv = b / r;
      }
      c_[j] = c;
      s_[j] = sv;
      h[j] = r;
      h[j + 1] = 0.0;
      const double gj = gp[j];
      gp[j] = c * gj;
      gp[j + 1] = -sv * gj;
      const double rn = fabs(gp[j + 1]);
      res[p] = rn;
      kcols[p] = j + 1;
      if (!(rn > target[p]) || sub == 0.0) active[p] = 0;
    }
    if (active[p]) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *any = s_any;
}

// y[p] = R_p^{-1} g[p] for each problem's kcols[p] x kcols[p] rotated Hessenberg
__global__ void k_seg_lsq(int32_t P, const double* __restrict__ H, int32_t ldh, int32_t m,
                          const int* __restrict__ kcols, const double* __restrict__ g, double* __restrict__ y) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int k = kcols[p];
    const double* Hp = H + (int64_t)p * ldh * m;
    const double* gp = g + (int64_t)p * ldh;
    double* yp = y + (int64_t)p * m;
    for (int i = k - 1; i >= 0; --i) {
      double s = gp[i];
      for (int jj = i + 1; jj < k; ++jj) s -= Hp[(int64_t)jj * ldh + i] * yp[jj];
      const double d = Hp[(int64_t)i * ldh + i];
      yp[i] = d != 0.0 ? s / d : 0.0;
    }
  }
}

// x_i += sum_{q < kcols[p(i)]} y[p(i)][q] Z_q[i]
__global__ void k_seg_update_x(SegDev sg, int64_t n, const double* __restrict__ Z, int64_t ldz,
                               const double* __restrict__ y, int32_t m, const int* __restrict__ kcols,
                               double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = sg.node_prob[i / 7];
    const int k = kcols[p];
    const double* yp = y + (int64_t)p * m;
    double s = x[i];
    for (int q = 0; q < k; ++q) s += yp[q] * Z[(int64_t)q * ldz + i];
    x[i] = s;
  }
}

// out_i = x_i + alpha[p(i)] y_i
__global__ void k_seg_axpy(SegDev sg, int64_t n, const double* __restrict__ x, const double* __restrict__ alpha,
                           const double* __restrict__ y, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = alpha[sg.node_prob[i / 7]];
    out[i] = a != 0.0 ? x[i] + a * y[i] : x[i];
  }
}

// out_i = mask[p(i)] ? 0 : -x_i
__global__ void k_seg_neg_masked(SegDev sg, int64_t n, const double* __restrict__ x, const int* __restrict__ mask,
                                 double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mask[sg.node_prob[i / 7]] ? 0.0 : -x[i];
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

inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = 152 * 32;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// groups of 8 vectors in one launch, then the partial last group (r vectors) in a
// launch of its own width
void mdot_groups(const SegDev& sg, int32_t n, const double* V, int64_t ldv, const double* w, double* partial,
                 double* out, int32_t ldo, int take_sqrt, int nself, const int* guard, cudaStream_t s) {
  const unsigned nch = (unsigned)sg.n_chunks;
  const int full = n / MD, r = n % MD;
  if (full > 0)
    k_seg_mdot<8, 2><<<dim3(nch, full), RB, 0, s>>>(sg, n, 0, V, ldv, w, partial, out, ldo, take_sqrt, nself, guard);
  if (r == 0) return;
  const dim3 g1(nch, 1);
  if (r == 1)
    k_seg_mdot<1, 8><<<g1, RB, 0, s>>>(sg, n, full, V, ldv, w, partial, out, ldo, take_sqrt, nself, guard);
  else if (r == 2)
    k_seg_mdot<2, 4><<<g1, RB, 0, s>>>(sg, n, full, V, ldv, w, partial, out, ldo, take_sqrt, nself, guard);
  else if (r <= 4)
    k_seg_mdot<4, 4><<<g1, RB, 0, s>>>(sg, n, full, V, ldv, w, partial, out, ldo, take_sqrt, nself, guard);
  else
    k_seg_mdot<8, 2><<<g1, RB, 0, s>>>(sg, n, full, V, ldv, w, partial, out, ldo, take_sqrt, nself, guard);
}

}  // namespace

int launch_seg_mdot(const SegDev& sg, int32_t nv, const double* V, int64_t ldv, const double* w, double* partial,
                    double* out, int32_t ldo, const int* guard, cudaStream_t s, int with_self) {
  const int n = nv + (with_self ? 1 : 0);
  mdot_groups(sg, n, V, ldv, w, partial, out, ldo, 0, with_self ? 1 : 0, guard, s);
  return (n / MD > 0 ? 1 : 0) + (n % MD > 0 ? 1 : 0);
}

void launch_seg_norm(const SegDev& sg, const double* x, double* partial, double* out, int32_t ldo,
                     const int* guard, cudaStream_t s) {
  mdot_groups(sg, 1, nullptr, 0, x, partial, out, ldo, 1, 0, guard, s);
}


void launch_seg_reorth_decide(int32_t P, const double* ws, const double* nrm, int32_t ldn, double* hb, int32_t lda,
                              int32_t j, const int* active, int* flag, cudaStream_t s) {
  k_seg_reorth_decide<<<1, 256, 0, s>>>(P, ws, nrm, ldn, hb, lda, j, active, flag);
}

void launch_seg_maxpy(const SegDev& sg, int64_t n, int32_t nv, const double* V, int64_t ldv, const double* h,
                      int32_t ldh, double* w, const int* guard, cudaStream_t s, const double* scal) {
  k_seg_maxpy<<<grid_for(n, 256), 256, 0, s>>>(sg, n, nv, V, ldv, h, ldh, w, scal, guard);
}

void launch_seg_norm_pythagoras(int32_t P, const double* hb, int32_t lda, int32_t j, double* hsub, int64_t ldsub,
                                double* inv, int* unsafe, int* flag, int force, const int* guard, cudaStream_t s) {
  k_seg_norm_pythagoras<<<1, 256, 0, s>>>(P, hb, lda, j, hsub, ldsub, inv, unsafe, flag, force, guard);
}

void launch_seg_norm_fix(int32_t P, const double* nrm, const int* unsafe, double* hsub, int64_t ldsub, double* scal,
                         const int* guard, cudaStream_t s) {
  k_seg_norm_fix<<<1, 256, 0, s>>>(P, nrm, unsafe, hsub, ldsub, scal, guard);
}

void launch_seg_scale_inv(const SegDev& sg, int64_t n, const double* x, const double* scal, int32_t lds,
                          double* y, const int* guard, cudaStream_t s) {
  k_seg_scale_inv<<<grid_for(n, 256), 256, 0, s>>>(sg, n, x, scal, lds, y, guard);
}

void launch_seg_cycle_init(int32_t P, double* g, int32_t ldg, const double* beta, const double* target, int* active,
                           int* kcols, int* any, cudaStream_t s) {
  k_seg_cycle_init<<<1, 256, 0, s>>>(P, g, ldg, beta, target, active, kcols, any);
}

void launch_seg_givens(int32_t P, const double* a, const double* b, int32_t lda, double* H, int32_t ldh, int32_t m,
                       int32_t j, double* cs, double* sn, double* g, double* res, const double* target, int* active,
                       int* kcols, int* any, cudaStream_t s) {
  k_seg_givens<<<1, 256, 0, s>>>(P, a, b, lda, H, ldh, m, j, cs, sn, g, res, target, active, kcols, any);
}

void launch_seg_lsq(int32_t P, const double* H, int32_t ldh, int32_t m, const int* kcols, const double* g, double* y,
                    cudaStream_t s) {
  k_seg_lsq<<<(P + 63) / 64, 64, 0, s>>>(P, H, ldh, m, kcols, g, y);
}

void launch_seg_update_x(const SegDev& sg, int64_t n, const double* Z, int64_t ldz, const double* y, int32_t m,
                         const int* kcols, double* x, cudaStream_t s) {
  k_seg_update_x<<<grid_for(n, 256), 256, 0, s>>>(sg, n, Z, ldz, y, m, kcols, x);
}

void launch_seg_axpy(const SegDev& sg, int64_t n, const double* x, const double* alpha, const double* y, double* out,
                     cudaStream_t s) {
  k_seg_axpy<<<grid_for(n, 256), 256, 0, s>>>(sg, n, x, alpha, y, out);
}

void launch_seg_neg_masked(const SegDev& sg, int64_t n, const double* x, const int* mask, double* out,
                           cudaStream_t s) {
  k_seg_neg_masked<<<grid_for(n, 256), 256, 0, s>>>(sg, n, x, mask, out);
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

}  // namespace fsi
