// Block-sparse (7x7 BSR) matrix-vector product and the restricted additive
// Schwarz preconditioner of Sec. 3, Eq. 14-16, with block ILU(k) subdomain
// solves: extraction of the overlapped submatrices J_i^delta, the batched
// factorisation (one CTA per subdomain, all subdomains in one launch), and the
// level-scheduled forward/backward solves with the restricted (owned-rows-only)
// prolongation used when the TMA-fed apply (ras_stream.cu) does not fit.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fsi {

namespace {

inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = 152 * 64;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ---------------------------------------------------------------------------
// SpMV: one warp per block row. Lane l < 28 owns output component r = l / 4 and
// every fourth block (q = l % 4) of the row; the four partial sums of a
// component are combined by two shuffles. Lanes 28..31 idle. FP64: values,
// vector and sums in FP64. Mixed: FP32 values and an FP32 copy of the vector;
// each block's 7-term product is formed in FP32 and the block products are
// accumulated in FP64 (one FP64 add per block and component), result in FP64.
// ---------------------------------------------------------------------------
template <class TV, class TX, int S>
__global__ void __launch_bounds__(256) k_bsr_spmv(int64_t n, const int64_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, const TV* __restrict__ vals,
                                                  const TX* __restrict__ x, double* __restrict__ y,
                                                  const int* __restrict__ guard) {
  // S block slots x 8 component lanes (7 used) per row; 32 / (8 S) rows per warp
  if (guard && *guard == 0) return;
  constexpr int G = 8 * S;
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int r = gl / S, q = gl % S;
  const int64_t grp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t base = grp0 - (lane / G); base < n; base += ngrp) {
    const int64_t row = base + (lane / G);
    double acc = 0.0;
    if (r < 7 && row < n) {
      const int64_t b0 = row_ptr[row], b1 = row_ptr[row + 1];
      // four of this lane's blocks per pass: their column indices first, then
      // all their loads, so that the loads of a pass are in flight together
      for (int64_t b = b0 + q; b < b1; b += 4 * S) {
        int cl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cl[u] = b + u * S < b1 ? col[b + u * S] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (cl[u] >= 0) {
            const TV* A = vals + 49 * (b + u * S) + 7 * r;
            const TX* xb = x + 7 * (int64_t)cl[u];
            TX s0 = TX(A[0]) * xb[0] + TX(A[1]) * xb[1];
            TX s1 = TX(A[2]) * xb[2] + TX(A[3]) * xb[3];
            TX s2 = TX(A[4]) * xb[4] + TX(A[5]) * xb[5];
            acc += (double)((s0 + s1) + (s2 + TX(A[6]) * xb[6]));
          }
        }
      }
    }
#pragma unroll
    for (int o = 1; o < S; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < 7 && q == 0 && row < n) y[7 * row + r] = acc;
  }
}

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y,
                           const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// ---------------------------------------------------------------------------
// RAS: extraction of J_i^delta = R_i^delta J (R_i^delta)^T (Eq. 15)
// ---------------------------------------------------------------------------
template <class TF, class TJ>
__global__ void k_ras_extract(int64_t nblocks, const int64_t* __restrict__ gblk, const TJ* __restrict__ vals,
                              TF* __restrict__ fac) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 49 * nblocks;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / 49;
    const int e = (int)(idx - 49 * b);
    const int64_t gb = gblk[b];
    fac[idx] = gb >= 0 ? (TF)vals[49 * gb + e] : TF(0);
  }
}

template <class TF> __device__ __forceinline__ TF tiny_pivot();
template <> __device__ __forceinline__ double tiny_pivot<double>() { return 1e-300; }
template <> __device__ __forceinline__ float tiny_pivot<float>() { return 1e-37f; }

// In-place inverse of the 7x7 block B (row-major) by one warp: Gauss-Jordan with
// partial pivoting on the augmented [B | I] in shared memory `aug` (7 x 14).
template <class TF>
__device__ void warp_invert7(TF* B, TF* aug, int32_t* err) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < 98; e += 32) {
    const int r = e / 14, c = e - 14 * r;
    aug[e] = c < 7 ? B[7 * r + c] : (c - 7 == r ? TF(1) : TF(0));
  }
  __syncwarp();
  for (int k = 0; k < 7; ++k) {
    // pivot search (lane 0), row swap
    int piv = k;
    if (lane == 0) {
      TF best = fabs(aug[14 * k + k]);
      for (int r = k + 1; r < 7; ++r) {
        TF v = fabs(aug[14 * r + k]);
        if (v > best) { best = v; piv = r; }
      }
      if (!(best > tiny_pivot<TF>())) atomicExch(err, 1);
    }
    piv = __shfl_sync(0xffffffffu, piv, 0);
    if (piv != k && lane < 14) {
      TF a = aug[14 * k + lane];
      aug[14 * k + lane] = aug[14 * piv + lane];
      aug[14 * piv + lane] = a;
    }
    __syncwarp();
    const TF inv = TF(1) / aug[14 * k + k];
    __syncwarp();
    if (lane < 14) aug[14 * k + lane] *= inv;
    __syncwarp();
    // every lane reads the multipliers of its entries before any lane writes
    TF fct[4];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = lane + 32 * it;
      fct[it] = e < 98 ? aug[14 * (e / 14) + k] : TF(0);
    }
    __syncwarp();
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = lane + 32 * it;
      if (e < 98) {
        const int r = e / 14, c = e - 14 * r;
        if (r != k) aug[e] -= fct[it] * aug[14 * k + c];
      }
    }
    __syncwarp();
  }
  for (int e = lane; e < 49; e += 32) {
    const int r = e / 7, c = e - 7 * r;
    B[e] = aug[14 * r + 7 + c];
  }
  __syncwarp();
}

// Batched block ILU, whole CTA on one row: one CTA per subdomain walks its rows
// in increasing order (a topological order of the elimination). At the start
// of a row the row itself is loaded into shared memory. For each L block (i,k):
// threads 0..48 form A_ik D_k^{-1} (D_k: the inverted pivot of the finished row
// k; into a separate buffer and the row), then all threads apply its updates
// A_ij -= A_ik A_kj (task = update x column) - two barriers per L block.
// MODE picks how much besides the row lives in shared memory, largest first
// (the factor_mode option of fsi_options is MODE + 1):
//   0: the pivots D_k of all L blocks of the row, loaded with the row, and the
//      source blocks A_kj of each L block's updates in a cp.async double
//      buffer, one L block ahead (their latency hides behind the previous L
//      block's arithmetic);
//   1: as 0 but D_k read from global memory (L2) when used;
//   2: only the row: D_k and the sources read from global memory when used.
// All three do the same arithmetic in the same order (bitwise identical
// factors); MODE 2 (factor_mode 3, the row only) is the default (see
// ras_factor_fits).
template <class TF>
__device__ __forceinline__ void cp_async_elem(TF* dst, const TF* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(sizeof(TF))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <class TF>
__device__ __forceinline__ void fetch_sources(const RasDev& R, const TF* fac, int64_t e, TF* buf, int tid, int nt) {
  const int64_t ub = R.upd_ptr[e];
  const int ne = (int)(R.upd_ptr[e + 1] - ub);
  for (int idx = tid; idx < 49 * ne; idx += nt) {
    const int u = idx / 49;
    cp_async_elem<TF>(buf + idx, fac + 49 * R.upd_src[ub + u] + (idx - 49 * u));
  }
}

template <class TF, int MODE>
__global__ void __launch_bounds__(256) k_ras_factor_cta(RasDev R, TF* __restrict__ fac, int32_t* err) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const size_t me = MODE <= 1 ? (size_t)R.max_entry_upd * 49 : 0;
  TF* sRow = reinterpret_cast<TF*>(fsm);
  TF* sD = sRow + (size_t)R.max_row_blocks * 49;
  TF* sSrc0 = sD + (MODE == 0 ? (size_t)R.max_row_lent * 49 : 0);
  TF* sSrc1 = sSrc0 + me;
  TF* sScl = sSrc1 + me;
  TF* sAug = sScl + 49;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int s = blockIdx.x;
  for (int64_t q = R.sd_row[s]; q < R.sd_row[s + 1]; ++q) {
    const int64_t rp = R.row_ptr[q];
    const int nblk = (int)(R.row_ptr[q + 1] - rp);
    const int64_t e0 = R.lent_ptr[q], e1 = R.lent_ptr[q + 1];
    const int nl = (int)(e1 - e0);
    if (MODE <= 1) {
      if (e0 < e1) fetch_sources<TF>(R, fac, e0, sSrc0, tid, nt);
      cp_async_commit();
    }
    for (int idx = tid; idx < 49 * nblk; idx += nt) sRow[idx] = fac[49 * rp + idx];
    if (MODE == 0)
      for (int idx = tid; idx < 49 * nl; idx += nt) {
        const int e = idx / 49;
        sD[idx] = fac[49 * R.lent_kdiag[e0 + e] + (idx - 49 * e)];
      }
    __syncthreads();
    for (int64_t e = e0; e < e1; ++e) {
      TF* cur = ((e - e0) & 1) ? sSrc1 : sSrc0;
      TF* nxt = ((e - e0) & 1) ? sSrc0 : sSrc1;
      if (MODE <= 1) {
        if (e + 1 < e1) fetch_sources<TF>(R, fac, e + 1, nxt, tid, nt);
        cp_async_commit();
      }
      TF* Aik = sRow + 49 * (R.lent_pos[e] - rp);
      if (tid < 49) {
        const TF* Dk = MODE == 0 ? sD + 49 * (e - e0) : fac + 49 * R.lent_kdiag[e];
        const int r = tid / 7, c = tid - 7 * r;
        TF v = TF(0);
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) v += Aik[7 * r + mm] * Dk[7 * mm + c];
        sScl[tid] = v;
      }
      if (MODE <= 1) cp_async_wait1();  // this thread's copies of L block e have landed
      __syncthreads();
      if (tid < 49) Aik[tid] = sScl[tid];
      const int64_t ub = R.upd_ptr[e];
      const int ntask = 7 * (int)(R.upd_ptr[e + 1] - ub);
      for (int t = tid; t < ntask; t += nt) {
        const int u = t / 7, cc = t - 7 * u;
        TF* Aij = sRow + 49 * (R.upd_tgt[ub + u] - rp) + cc;
        const TF* Akj = (MODE <= 1 ? cur + 49 * u : fac + 49 * R.upd_src[ub + u]) + cc;
        TF col[7];
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) col[mm] = Akj[7 * mm];
#pragma unroll
        for (int rr = 0; rr < 7; ++rr) {
          TF acc = Aij[7 * rr];
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) acc -= sScl[7 * rr + mm] * col[mm];
          Aij[7 * rr] = acc;
        }
      }
      __syncthreads();
    }
    if (tid < 32) warp_invert7<TF>(sRow + 49 * (R.diag[q] - rp), sAug, err);
    __syncthreads();
    for (int idx = tid; idx < 49 * nblk; idx += nt) fac[49 * rp + idx] = sRow[idx];
    __syncthreads();
  }
}

// Block ILU on nested-dissection ordered subdomains: the CTA's 256 threads
// form G = 2^D groups (D the subdomain's dissection depth); in each phase (the
// leaves, then the separators level by level) every item of the phase is
// factored by its own group, row by row exactly as MODE 2 of k_ras_factor_cta
// does it (the row in shared memory, pivots and sources read from global
// memory), with the group's own barrier instead of the CTA's. Items of one
// phase share no entry, so their rows can be eliminated side by side; the
// arithmetic of every row is that of the sequential kernel, in the same order
// (bitwise identical factors). A CTA barrier separates the phases.
__device__ __forceinline__ void group_sync(int g, int gs) {
  if (gs == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(gs) : "memory");
  }
}

template <class TF>
__global__ void __launch_bounds__(256) k_ras_factor_nd(RasDev R, TF* __restrict__ fac, int32_t* err) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int s = blockIdx.x;
  const int D = R.sd_depth[s];
  const int G = 1 << D, gs = blockDim.x / G;
  const int g = threadIdx.x / gs, lt = threadIdx.x - g * gs;
  const size_t per = (size_t)(R.max_row_blocks + 1) * 49 + 98;
  TF* sRow = reinterpret_cast<TF*>(fsm) + (size_t)g * per;
  TF* sScl = sRow + (size_t)R.max_row_blocks * 49;
  TF* sAug = sScl + 49;
  const int64_t r0 = R.sd_row[s];
  const int64_t* irow = R.item_row + R.sd_item[s];
  for (int p = 0; p <= D; ++p) {
    const int nit = 1 << (D - p);
    if (g < nit) {
      const int it = (1 << (D + 1)) - (1 << (D - p + 1)) + g;
      const int64_t qb = r0 + (it == 0 ? 0 : irow[it - 1]), qe = r0 + irow[it];
      for (int64_t q = qb; q < qe; ++q) {
        const int64_t rp = R.row_ptr[q];
        const int nblk = (int)(R.row_ptr[q + 1] - rp);
        const int64_t e0 = R.lent_ptr[q], e1 = R.lent_ptr[q + 1];
        for (int idx = lt; idx < 49 * nblk; idx += gs) sRow[idx] = fac[49 * rp + idx];
        group_sync(g, gs);
        for (int64_t e = e0; e < e1; ++e) {
          TF* Aik = sRow + 49 * (R.lent_pos[e] - rp);
          const TF* Dk = fac + 49 * R.lent_kdiag[e];
          for (int x = lt; x < 49; x += gs) {
            const int r = x / 7, c = x - 7 * r;
            TF v = TF(0);
#pragma unroll
            for (int mm = 0; mm < 7; ++mm) v += Aik[7 * r + mm] * Dk[7 * mm + c];
            sScl[x] = v;
          }
          group_sync(g, gs);
          for (int x = lt; x < 49; x += gs) Aik[x] = sScl[x];
          const int64_t ub = R.upd_ptr[e];
          const int ntask = 7 * (int)(R.upd_ptr[e + 1] - ub);
          for (int t = lt; t < ntask; t += gs) {
            const int u = t / 7, cc = t - 7 * u;
            TF* Aij = sRow + 49 * (R.upd_tgt[ub + u] - rp) + cc;
            const TF* Akj = fac + 49 * R.upd_src[ub + u] + cc;
            TF col[7];
#pragma unroll
            for (int mm = 0; mm < 7; ++mm) col[mm] = Akj[7 * mm];
#pragma unroll
            for (int rr = 0; rr < 7; ++rr) {
              TF acc = Aij[7 * rr];
#pragma unroll
              for (int mm = 0; mm < 7; ++mm) acc -= sScl[7 * rr + mm] * col[mm];
              Aij[7 * rr] = acc;
            }
          }
          group_sync(g, gs);
        }
        if (lt < 32) warp_invert7<TF>(sRow + 49 * (R.diag[q] - rp), sAug, err);
        group_sync(g, gs);
        for (int idx = lt; idx < 49 * nblk; idx += gs) fac[49 * rp + idx] = sRow[idx];
        group_sync(g, gs);
      }
    }
    __syncthreads();
  }
}

// Batched RAS apply: grid = one CTA per subdomain; 8-lane groups own one row
// (lane c < 7 computes component c). work holds the subdomain vector.
template <class TF>
__global__ void __launch_bounds__(256) k_ras_apply(RasDev R, const TF* __restrict__ fac,
                                                   const double* __restrict__ rin, TF* __restrict__ work,
                                                   double* __restrict__ z, float* __restrict__ z32,
                                                   const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  const int s = blockIdx.x;
  const int64_t r0 = R.sd_row[s], m = R.sd_row[s + 1] - r0;
  const int grp = threadIdx.x >> 3, c = threadIdx.x & 7;
  const int ngrp = blockDim.x >> 3;
  TF* w = work + 7 * r0;
  // restriction R_i^delta r
  for (int64_t idx = threadIdx.x; idx < 7 * m; idx += blockDim.x) {
    const int64_t q = idx / 7;
    const int cc = (int)(idx - 7 * q);
    w[idx] = (TF)rin[7 * (int64_t)R.gnode[r0 + q] + cc];
  }
  __syncthreads();
  // forward solve with the unit lower factor
  for (int64_t l = R.sd_lvlL[s]; l < R.sd_lvlL[s + 1]; ++l) {
    const int64_t lb = R.lvlL_ptr[l], le = R.lvlL_ptr[l + 1];
    for (int64_t ri = lb + grp; ri < le; ri += ngrp) {
      const int64_t q = R.lvlL_rows[ri];
      const int64_t gq = r0 + q;
      if (c < 7) {
        TF acc = w[7 * q + c];
        for (int64_t e = R.row_ptr[gq]; e < R.diag[gq]; ++e) {
          const TF* A = fac + 49 * e + 7 * c;
          const TF* xk = work + 7 * (int64_t)R.col[e];
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) acc -= A[mm] * xk[mm];
        }
        w[7 * q + c] = acc;
      }
    }
    __syncthreads();
  }
  // backward solve with the upper factor and inverted pivots
  for (int64_t l = R.sd_lvlU[s]; l < R.sd_lvlU[s + 1]; ++l) {
    const int64_t lb = R.lvlU_ptr[l], le = R.lvlU_ptr[l + 1];
    // rounds are uniform across the warp so that every lane joins the shuffles
    for (int64_t base = lb; base < le; base += ngrp) {
      const int64_t ri = base + grp;
      const bool act = ri < le;
      const int64_t q = act ? R.lvlU_rows[ri] : 0;
      const int64_t gq = r0 + q;
      TF acc = TF(0);
      if (act && c < 7) {
        acc = w[7 * q + c];
        for (int64_t e = R.diag[gq] + 1; e < R.row_ptr[gq + 1]; ++e) {
          const TF* A = fac + 49 * e + 7 * c;
          const TF* xk = work + 7 * (int64_t)R.col[e];
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) acc -= A[mm] * xk[mm];
        }
      }
      // z_q = D_q^{-1} t: gather t from the 7 lanes of the group
      TF tv[7];
#pragma unroll
      for (int mm = 0; mm < 7; ++mm) tv[mm] = __shfl_sync(0xffffffffu, acc, (threadIdx.x & 31 & ~7) + mm);
      if (act && c < 7) {
        const TF* Dinv = fac + 49 * R.diag[gq] + 7 * c;
        TF zz = TF(0);
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) zz += Dinv[mm] * tv[mm];
        w[7 * q + c] = zz;
      }
    }
    __syncthreads();
  }
  // restricted prolongation (R_i^0)^T: owned rows only
  for (int64_t idx = threadIdx.x; idx < 7 * m; idx += blockDim.x) {
    const int64_t q = idx / 7;
    const int cc = (int)(idx - 7 * q);
    if (R.owned[r0 + q]) {
      z[7 * (int64_t)R.gnode[r0 + q] + cc] = (double)w[idx];
      if (z32) z32[7 * (int64_t)R.gnode[r0 + q] + cc] = (float)w[idx];
    }
  }
}

}  // namespace

template <class TV, class TX>
void launch_bsr_spmv(int64_t n, const int64_t* row_ptr, const int32_t* col, const TV* vals, const TX* x,
                     double* y, int threads_per_row, const int* guard, cudaStream_t s) {
  if (threads_per_row == 16)
    k_bsr_spmv<TV, TX, 2><<<grid_for(16 * n, 256), 256, 0, s>>>(n, row_ptr, col, vals, x, y, guard);
  else
    k_bsr_spmv<TV, TX, 4><<<grid_for(32 * n, 256), 256, 0, s>>>(n, row_ptr, col, vals, x, y, guard);
}

void launch_to_float(int64_t n, const double* x, float* y, const int* guard, cudaStream_t s) {
  k_to_float<<<grid_for(n, 256), 256, 0, s>>>(n, x, y, guard);
}

template <class TF, class TJ>
void launch_ras_extract(const RasDev& r, const TJ* vals, TF* fac, cudaStream_t s) {
  k_ras_extract<TF, TJ><<<grid_for(49 * r.nblocks, 256), 256, 0, s>>>(r.nblocks, r.gblk, vals, fac);
}

template <class TF>
size_t ras_factor_cta_smem(const RasDev& r, int mode) {
  if (mode == 3)  // one row, scaled block and inversion scratch per group
    return ((size_t)1 << r.max_depth) * (((size_t)r.max_row_blocks + 1) * 49 + 98) * sizeof(TF);
  size_t blocks = (size_t)r.max_row_blocks + 1;  // the row and the scaled L block
  if (mode == 0) blocks += (size_t)r.max_row_lent + 2 * (size_t)r.max_entry_upd;
  if (mode == 1) blocks += 2 * (size_t)r.max_entry_upd;
  return (blocks * 49 + 98) * sizeof(TF);  // + the 7 x 14 inversion scratch
}

// Fit check of a factorisation mode. The automatic choice is the leanest mode
// (2): measured on GB300 it is the fastest, because the smaller footprint lets
// more subdomain CTAs share an SM, which hides the latency of the pivot and
// source reads better than prefetching them does.
template <class TF>
bool ras_factor_fits(const RasDev& r, int mode) {
  return ras_factor_cta_smem<TF>(r, mode) <= FACTOR_SMEM_MAX;
}

template <class TF, int MODE>
void launch_factor_mode(const RasDev& r, TF* fac, int32_t* err, size_t smem, cudaStream_t s) {
  cudaFuncSetAttribute(k_ras_factor_cta<TF, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_ras_factor_cta<TF, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ras_factor_cta<TF, MODE><<<r.np, 256, smem, s>>>(r, fac, err);
}

template <class TF>
void launch_ras_factor(const RasDev& r, TF* fac, int32_t* err, cudaStream_t s) {
  const size_t smem = ras_factor_cta_smem<TF>(r, r.factor_mode);
  switch (r.factor_mode) {
    case 0: launch_factor_mode<TF, 0>(r, fac, err, smem, s); break;
    case 1: launch_factor_mode<TF, 1>(r, fac, err, smem, s); break;
    case 2: launch_factor_mode<TF, 2>(r, fac, err, smem, s); break;
    case 3:
      cudaFuncSetAttribute(k_ras_factor_nd<TF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
      cudaFuncSetAttribute(k_ras_factor_nd<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ras_factor_nd<TF><<<r.np, 256, smem, s>>>(r, fac, err);
      break;
    default: break;  // fsi_create rejects such plans
  }
}

template bool ras_factor_fits<float>(const RasDev&, int);
template bool ras_factor_fits<double>(const RasDev&, int);

template <class TF>
void launch_ras_apply(const RasDev& r, const TF* fac, const double* rin, TF* work, double* z, float* z32,
                      const int* guard, cudaStream_t s) {
  k_ras_apply<TF><<<r.np, 256, 0, s>>>(r, fac, rin, work, z, z32, guard);
}

template void launch_bsr_spmv<double, double>(int64_t, const int64_t*, const int32_t*, const double*,
                                              const double*, double*, int, const int*, cudaStream_t);
template void launch_bsr_spmv<float, float>(int64_t, const int64_t*, const int32_t*, const float*, const float*,
                                            double*, int, const int*, cudaStream_t);
template void launch_ras_extract<double, double>(const RasDev&, const double*, double*, cudaStream_t);
template void launch_ras_extract<float, float>(const RasDev&, const float*, float*, cudaStream_t);
template void launch_ras_factor<double>(const RasDev&, double*, int32_t*, cudaStream_t);
template void launch_ras_factor<float>(const RasDev&, float*, int32_t*, cudaStream_t);
template void launch_ras_apply<double>(const RasDev&, const double*, const double*, double*, double*, float*,
                                       const int*, cudaStream_t);
template void launch_ras_apply<float>(const RasDev&, const float*, const double*, float*, double*, float*,
                                      const int*, cudaStream_t);

}  // namespace fsi
