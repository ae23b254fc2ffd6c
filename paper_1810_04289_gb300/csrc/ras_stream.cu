// Streamed RAS apply (Sec. 3, Eq. 16) for GB300: one CTA per subdomain, two
// warps. Warp 1 (one elected lane) is a producer that streams the packed factor
// with 1-D bulk copies (cp.async.bulk, the TMA engine) into a ring of
// shared-memory stages guarded by mbarriers; warp 0 is the consumer that walks
// the rows in order (forward solve with the unit lower factor, then backward
// solve with the upper factor and inverted pivots) on the subdomain vector held
// in shared memory. The dependency chain of an ILU solve on an RCM-ordered
// subdomain is nearly the row count, so the rows are processed one after the
// other by 28 lanes (4 blocks at a time x 7 components) while the factor bytes
// for the rows ahead are already in flight.
//
// Packed layout (built by k_pack_factors after each factorisation):
//   L stream: for every row in increasing order, its L blocks;
//   U stream: for every row in decreasing order, its inverted pivot, then its U blocks.
// Each packed block holds 49 values, then the subdomain-relative column row in
// the first 4 bytes of slot 49, padded to a 16-byte multiple (52 floats, 50 doubles).
// Stages are fixed slices of stage_blocks blocks of a subdomain's L stream, then
// of its U stream; a row may straddle stages (its partial sums carry over), so
// the stage size is independent of the row length and can be chosen for
// occupancy.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records
// FSI_ERR_TIMEOUT-style status in *err, drains (bounded) and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace fsi {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: returns false if the barrier phase did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 20); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <class TF> struct Pack;
template <> struct Pack<float> { static constexpr int stride = 52; };
template <> struct Pack<double> { static constexpr int stride = 50; };

template <class TF>
__device__ __forceinline__ int blk_col(const TF* blk) {
  return *reinterpret_cast<const int*>(blk + 49);
}

constexpr int NSTMAX = 8;  // most ring stages (runtime count R.nst)

// sum over blocks b in [b0, nb) of (block b, row c) . w[col(b)], reduced over
// the warp: lane = 7 j + c handles blocks b0 + j, b0 + j + 4, ...; every block
// gathers its column index first so that all loads of a chunk are independent,
// then forms the 7-term products as a short tree. The total lands in lanes 0..6.
template <class TF, int STR>
__device__ __forceinline__ TF row_dot(const TF* stg, int b0, int nb, const TF* w, int j, int c) {
  TF acc = TF(0);
  if (j < 4) {
    for (int b = b0 + j; b < nb; b += 16) {
      int cols[4];
      const TF* blk[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int bi = b + 4 * i;
        blk[i] = stg + (size_t)(bi < nb ? bi : b) * STR;
        cols[i] = bi < nb ? blk_col(blk[i]) : -1;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (cols[i] >= 0) {
          const TF* a = blk[i] + 7 * c;
          const TF* x = w + 7 * cols[i];
          const TF p01 = a[0] * x[0] + a[1] * x[1];
          const TF p23 = a[2] * x[2] + a[3] * x[3];
          const TF p45 = a[4] * x[4] + a[5] * x[5];
          acc += (p01 + p23) + (p45 + a[6] * x[6]);
        }
      }
    }
  }
  acc += __shfl_down_sync(0xffffffffu, acc, 14);
  acc += __shfl_down_sync(0xffffffffu, acc, 7);
  return acc;
}

template <class TF>
__global__ void __launch_bounds__(64) k_ras_apply_stream(RasStreamDev R, const double* __restrict__ rin,
                                                         double* __restrict__ z, float* __restrict__ z32,
                                                         int32_t* err, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  constexpr int STR = Pack<TF>::stride;
  extern __shared__ __align__(128) unsigned char smem[];
  const int NST = R.nst;
  const int SB = R.stage_blocks;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + NSTMAX;
  TF* ring = reinterpret_cast<TF*>(smem + 128);
  TF* w = ring + (size_t)NST * SB * STR;
  const int s = blockIdx.x;
  const int64_t r0 = R.sd_row[s];
  const int m = (int)(R.sd_row[s + 1] - r0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-row block counts of both streams, next to the vector
  unsigned short* Lcnt = reinterpret_cast<unsigned short*>(w + 7 * (size_t)R.max_rows);
  unsigned short* Ucnt = Lcnt + R.max_rows;
  const int64_t Lb0 = R.L_off[s], Ub0 = R.U_off[s];
  const int64_t nLb = R.L_off[s + 1] - Lb0, nUb = R.U_off[s + 1] - Ub0;
  const int nGL = (int)((nLb + SB - 1) / SB);
  const int ngroups = nGL + (int)((nUb + SB - 1) / SB);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // restriction R_i^delta r into shared memory
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const double* src = rin + 7 * (int64_t)R.gnode[r0 + q];
    double v[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) v[c] = src[c];
#pragma unroll
    for (int c = 0; c < 7; ++c) w[7 * q + c] = (TF)v[c];
    Lcnt[q] = (unsigned short)R.L_cnt[r0 + q];
    Ucnt[q] = (unsigned short)R.U_cnt[r0 + q];
  }
  __syncthreads();

  const TF* Lpack = reinterpret_cast<const TF*>(R.Lpack) + (size_t)Lb0 * STR;
  const TF* Upack = reinterpret_cast<const TF*>(R.Upack) + (size_t)Ub0 * STR;

  if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int it = 0;
      for (; it < ngroups && !R.stall; ++it) {
        const int st = it % NST;
        if (it >= NST) ok = mbar_wait(&empty[st], ((it / NST) - 1) & 1);
        if (!ok) break;
        const bool isL = it < nGL;
        const int64_t first = (int64_t)(isL ? it : it - nGL) * SB;
        const int64_t nb = (isL ? nLb : nUb) - first;
        const uint32_t bytes = (uint32_t)((nb < SB ? nb : SB) * STR * sizeof(TF));
        mbar_arrive_expect_tx(&full[st], bytes);
        bulk_g2s(ring + (size_t)st * SB * STR, (isL ? Lpack : Upack) + (size_t)first * STR, bytes, &full[st]);
      }
      if (!ok) atomicExch(err, 2);
      // drain: the last copy issued into each stage must land before the CTA
      // may exit (bounded; on the normal path these phases completed already)
      for (int k = (it > NST ? it - NST : 0); k < it; ++k) mbar_wait(&full[k % NST], (k / NST) & 1);
    }
    return;
  }

  // consumer warp. Per stage: finish the row that straddles in from the previous
  // stage, then the rows that lie wholly inside the stage (the common case, no
  // bookkeeping), then start the row that straddles out; its partial sum carries.
  const int j = lane / 7, c = lane - 7 * (lane / 7);  // block slot 0..3 (4 = idle), component
  bool ok = true;
  int it = 0;
  // forward: w_q -= sum_k L_qk w_k
  {
    int q = 0, rem = 0;
    TF acc = TF(0);
    for (int g = 0; g < nGL; ++g, ++it) {
      const int st = it % NST;
      ok = mbar_wait(&full[st], (it / NST) & 1);
      if (!ok) break;
      const TF* stg = ring + (size_t)st * SB * STR;
      const int cap = (int)min((int64_t)SB, nLb - (int64_t)g * SB);
      int pos = 0;
      if (rem > 0) {
        const int k = min(rem, cap);
        acc += row_dot<TF, STR>(stg, 0, k, w, j, c);
        pos = k;
        rem -= k;
        if (rem == 0) {
          if (lane < 7) w[7 * q + lane] -= acc;
          __syncwarp();
          ++q;
        }
      }
      if (rem == 0) {
        for (; q < m; ++q) {
          const int nb = Lcnt[q];
          if (pos + nb > cap) break;
          const TF a = row_dot<TF, STR>(stg + (size_t)pos * STR, 0, nb, w, j, c);
          if (lane < 7 && nb > 0) w[7 * q + lane] -= a;
          __syncwarp();
          pos += nb;
        }
        if (q < m && pos < cap) {
          acc = row_dot<TF, STR>(stg + (size_t)pos * STR, 0, cap - pos, w, j, c);
          rem = Lcnt[q] - (cap - pos);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  // backward: w_q = D_q^{-1} (w_q - sum_j U_qj w_j); the pivot is the row's first block
  if (ok) {
    int q = m - 1, rem = 0;
    TF acc = TF(0);
    TF dreg[7];
    auto finish = [&](int row, TF sum) {
      const TF t = (lane < 7) ? w[7 * row + lane] - sum : TF(0);
      TF tv[7];
#pragma unroll
      for (int mm = 0; mm < 7; ++mm) tv[mm] = __shfl_sync(0xffffffffu, t, mm);
      if (lane < 7) {
        TF zz = TF(0);
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) zz += dreg[mm] * tv[mm];
        w[7 * row + lane] = zz;
      }
      __syncwarp();
    };
    auto load_pivot = [&](const TF* blk) {
#pragma unroll
      for (int mm = 0; mm < 7; ++mm) dreg[mm] = lane < 7 ? blk[7 * lane + mm] : TF(0);
    };
    for (; it < ngroups; ++it) {
      const int st = it % NST;
      ok = mbar_wait(&full[st], (it / NST) & 1);
      if (!ok) break;
      const TF* stg = ring + (size_t)st * SB * STR;
      const int cap = (int)min((int64_t)SB, nUb - (int64_t)(it - nGL) * SB);
      int pos = 0;
      if (rem > 0) {
        const int k = min(rem, cap);
        acc += row_dot<TF, STR>(stg, 0, k, w, j, c);
        pos = k;
        rem -= k;
        if (rem == 0) {
          finish(q, acc);
          --q;
        }
      }
      if (rem == 0) {
        for (; q >= 0; --q) {
          const int nb = Ucnt[q];
          if (pos + nb > cap) break;
          const TF* rs = stg + (size_t)pos * STR;
          load_pivot(rs);
          finish(q, row_dot<TF, STR>(rs, 1, nb, w, j, c));
          pos += nb;
        }
        if (q >= 0 && pos < cap) {
          const TF* rs = stg + (size_t)pos * STR;
          load_pivot(rs);
          acc = row_dot<TF, STR>(rs, 1, cap - pos, w, j, c);
          rem = Ucnt[q] - (cap - pos);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  if (!ok) {
    if (lane == 0) atomicExch(err, 2);
    return;
  }
  // restricted prolongation (R_i^0)^T: owned rows only, one row per lane
  for (int q = lane; q < m; q += 32) {
    if (R.owned[r0 + q]) {
      const int64_t g7 = 7 * (int64_t)R.gnode[r0 + q];
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) z[g7 + cc] = (double)w[7 * q + cc];
      if (z32) {
#pragma unroll
        for (int cc = 0; cc < 7; ++cc) z32[g7 + cc] = (float)w[7 * q + cc];
      }
    }
  }
}

// copy the factor blocks into the packed streams
template <class TF>
__global__ void k_pack_factors(int64_t nL, const int64_t* __restrict__ Lsrc, const int32_t* __restrict__ Lcol,
                               int64_t nU, const int64_t* __restrict__ Usrc, const int32_t* __restrict__ Ucol,
                               const TF* __restrict__ fac, TF* __restrict__ Lpack, TF* __restrict__ Upack) {
  constexpr int STR = Pack<TF>::stride;
  const int64_t total = (nL + nU) * STR;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / STR;
    const int e = (int)(idx - STR * b);
    const bool isL = b < nL;
    const int64_t bb = isL ? b : b - nL;
    const int64_t src = isL ? Lsrc[bb] : Usrc[bb];
    TF* dst = (isL ? Lpack : Upack) + bb * STR;
    if (e < 49) {
      dst[e] = fac[49 * src + e];
    } else if (e == 49) {
      TF v = TF(0);
      *reinterpret_cast<int*>(&v) = isL ? Lcol[bb] : Ucol[bb];
      dst[e] = v;
    } else {
      dst[e] = TF(0);
    }
  }
}

}  // namespace

template <class TF>
size_t ras_stream_smem(const RasStreamDev& r) {
  return 128 + (size_t)r.nst * r.stage_blocks * Pack<TF>::stride * sizeof(TF) + (size_t)7 * r.max_rows * sizeof(TF) +
         (size_t)4 * r.max_rows + 16;
}

template <class TF>
void launch_pack_factors(const RasStreamDev& r, const TF* fac, cudaStream_t s) {
  const int64_t total = (r.nL + r.nU) * Pack<TF>::stride;
  int64_t g = (total + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_pack_factors<TF><<<(int)g, 256, 0, s>>>(r.nL, r.Lsrc, r.Lcol, r.nU, r.Usrc, r.Ucol, fac, (TF*)r.Lpack,
                                            (TF*)r.Upack);
}

template <class TF>
cudaError_t ras_stream_init(const RasStreamDev& r) {
  // all of the unified L1/shared storage as shared memory: several CTAs per SM
  cudaError_t e = cudaFuncSetAttribute(k_ras_apply_stream<TF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ras_apply_stream<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ras_stream_smem<TF>(r));
}

template <class TF>
cudaError_t launch_ras_apply_stream(const RasStreamDev& r, const double* rin, double* z, float* z32, int32_t* err,
                                    const int* guard, cudaStream_t s) {
  k_ras_apply_stream<TF><<<r.np, 64, ras_stream_smem<TF>(r), s>>>(r, rin, z, z32, err, guard);
  return cudaGetLastError();
}

template cudaError_t ras_stream_init<float>(const RasStreamDev&);
template cudaError_t ras_stream_init<double>(const RasStreamDev&);

template size_t ras_stream_smem<float>(const RasStreamDev&);
template size_t ras_stream_smem<double>(const RasStreamDev&);
template void launch_pack_factors<float>(const RasStreamDev&, const float*, cudaStream_t);
template void launch_pack_factors<double>(const RasStreamDev&, const double*, cudaStream_t);
template cudaError_t launch_ras_apply_stream<float>(const RasStreamDev&, const double*, double*, float*, int32_t*,
                                                    const int*, cudaStream_t);
template cudaError_t launch_ras_apply_stream<double>(const RasStreamDev&, const double*, double*, float*, int32_t*,
                                                     const int*, cudaStream_t);

}  // namespace fsi
