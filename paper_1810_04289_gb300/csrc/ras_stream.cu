// Streamed RAS apply (Sec. 3, Eq. 16) for GB300: one CTA per subdomain, two
// warps. Warp 1 (one elected lane) is a producer that streams the packed factor
// rows with 1-D bulk copies (cp.async.bulk, the TMA engine) into a ring of
// shared-memory stages guarded by mbarriers; warp 0 is the consumer that walks
// the rows in order (forward solve with the unit lower factor, then backward
// solve with the upper factor and inverted pivots) on the subdomain vector held
// in shared memory. The dependency chain of an ILU solve on an RCM-ordered
// subdomain is nearly the row count, so the rows are processed one after the
// other by all 28 lanes (4 blocks at a time x 7 components) while the factor
// bytes for the rows ahead are already in flight.
//
// Packed layout (built by k_pack_factors after each factorisation):
//   L stream: for every row in increasing order, its L blocks;
//   U stream: for every row in decreasing order, its inverted pivot, then its U blocks.
// Each packed block holds 49 values, then the subdomain-relative column row in
// the first 4 bytes of slot 49, padded to a 16-byte multiple (52 floats, 50 doubles).
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

constexpr int NST = 4;  // ring stages

// Each stage carries a group of consecutive rows of one stream (at most
// stage_blocks blocks), so one bulk copy moves several rows and NST groups are
// in flight ahead of the consumer.
template <class TF>
__global__ void __launch_bounds__(64) k_ras_apply_stream(RasStreamDev R, const double* __restrict__ rin,
                                                         double* __restrict__ z, int32_t* err) {
  constexpr int STR = Pack<TF>::stride;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + NST;
  TF* ring = reinterpret_cast<TF*>(smem + 128);
  TF* w = ring + (size_t)NST * R.stage_blocks * STR;
  const int s = blockIdx.x;
  const int64_t r0 = R.sd_row[s];
  const int m = (int)(R.sd_row[s + 1] - r0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // restriction R_i^delta r into shared memory
  for (int idx = threadIdx.x; idx < 7 * m; idx += blockDim.x) {
    const int q = idx / 7, c = idx - 7 * q;
    w[idx] = (TF)rin[7 * (int64_t)R.gnode[r0 + q] + c];
  }
  __syncthreads();

  const int64_t* Lcnt = R.L_cnt + r0;
  const int64_t* Ucnt = R.U_cnt + r0;
  const TF* Lpack = reinterpret_cast<const TF*>(R.Lpack);
  const TF* Upack = reinterpret_cast<const TF*>(R.Upack);
  const int64_t gL0 = R.gL_ptr[s], gL1 = R.gL_ptr[s + 1];
  const int64_t gU0 = R.gU_ptr[s], gU1 = R.gU_ptr[s + 1];
  const int ngroups = (int)((gL1 - gL0) + (gU1 - gU0));

  if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int it = 0;
      for (; it < ngroups; ++it) {
        const bool isL = it < gL1 - gL0;
        const int64_t g = isL ? gL0 + it : gU0 + (it - (gL1 - gL0));
        const int st = it % NST;
        if (it >= NST) ok = mbar_wait(&empty[st], ((it / NST) - 1) & 1);
        if (!ok) break;
        const int64_t nb = isL ? R.gL_nblk[g] : R.gU_nblk[g];
        const uint32_t bytes = (uint32_t)(nb * STR * sizeof(TF));
        mbar_arrive_expect_tx(&full[st], bytes);
        if (bytes) {
          const TF* src = (isL ? Lpack + (size_t)R.gL_blk[g] * STR : Upack + (size_t)R.gU_blk[g] * STR);
          bulk_g2s(ring + (size_t)st * R.stage_blocks * STR, src, bytes, &full[st]);
        }
      }
      if (!ok) atomicExch(err, 2);
      // drain: the last copy issued into each stage must land before the CTA
      // may exit (bounded; on the normal path these phases completed already)
      for (int k = (it > NST ? it - NST : 0); k < it; ++k) mbar_wait(&full[k % NST], (k / NST) & 1);
    }
    return;
  }

  // consumer warp
  const int j = lane / 7, c = lane - 7 * (lane / 7);  // block slot 0..3 (4 = idle), component
  bool ok = true;
  int it = 0;
  // forward: w_q -= sum_k L_qk w_k
  for (int64_t g = gL0; g < gL1 && ok; ++g, ++it) {
    const int st = it % NST;
    ok = mbar_wait(&full[st], (it / NST) & 1);
    if (!ok) break;
    const TF* stg = ring + (size_t)st * R.stage_blocks * STR;
    const int qa = R.gL_row[g];
    const int qend = (g + 1 < gL1) ? R.gL_row[g + 1] : m;   // exclusive, ascending
    for (int q = qa; q < qend; ++q) {
      const int nb = (int)Lcnt[q];
      TF acc0 = TF(0), acc1 = TF(0);
      if (j < 4) {
        int b = j;
        for (; b + 4 < nb; b += 8) {
          const TF* b0 = stg + (size_t)b * STR;
          const TF* b1 = b0 + 4 * STR;
          const TF* x0 = w + 7 * blk_col(b0);
          const TF* x1 = w + 7 * blk_col(b1);
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) {
            acc0 += b0[7 * c + mm] * x0[mm];
            acc1 += b1[7 * c + mm] * x1[mm];
          }
        }
        if (b < nb) {
          const TF* b0 = stg + (size_t)b * STR;
          const TF* x0 = w + 7 * blk_col(b0);
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) acc0 += b0[7 * c + mm] * x0[mm];
        }
      }
      TF acc = acc0 + acc1;
      acc += __shfl_down_sync(0xffffffffu, acc, 14);
      acc += __shfl_down_sync(0xffffffffu, acc, 7);
      if (lane < 7 && nb > 0) w[7 * q + lane] -= acc;
      __syncwarp();
      stg += (size_t)nb * STR;
    }
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  // backward: w_q = D_q^{-1} (w_q - sum_j U_qj w_j)
  for (int64_t g = gU0; g < gU1 && ok; ++g, ++it) {
    const int st = it % NST;
    ok = mbar_wait(&full[st], (it / NST) & 1);
    if (!ok) break;
    const TF* stg = ring + (size_t)st * R.stage_blocks * STR;
    const int qa = R.gU_row[g];                                // first (highest) row of the group
    const int qend = (g + 1 < gU1) ? R.gU_row[g + 1] : -1;     // exclusive, descending
    for (int q = qa; q > qend; --q) {
      const int nb = (int)Ucnt[q];
      TF acc0 = TF(0), acc1 = TF(0);
      if (j < 4) {
        int b = 1 + j;
        for (; b + 4 < nb; b += 8) {
          const TF* b0 = stg + (size_t)b * STR;
          const TF* b1 = b0 + 4 * STR;
          const TF* x0 = w + 7 * blk_col(b0);
          const TF* x1 = w + 7 * blk_col(b1);
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) {
            acc0 += b0[7 * c + mm] * x0[mm];
            acc1 += b1[7 * c + mm] * x1[mm];
          }
        }
        if (b < nb) {
          const TF* b0 = stg + (size_t)b * STR;
          const TF* x0 = w + 7 * blk_col(b0);
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) acc0 += b0[7 * c + mm] * x0[mm];
        }
      }
      TF acc = acc0 + acc1;
      acc += __shfl_down_sync(0xffffffffu, acc, 14);
      acc += __shfl_down_sync(0xffffffffu, acc, 7);
      const TF t = (lane < 7) ? w[7 * q + lane] - acc : TF(0);
      TF tv[7];
#pragma unroll
      for (int mm = 0; mm < 7; ++mm) tv[mm] = __shfl_sync(0xffffffffu, t, mm);
      if (lane < 7) {
        const TF* D = stg + 7 * lane;  // first block of the row: inverted pivot
        TF zz = TF(0);
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) zz += D[mm] * tv[mm];
        w[7 * q + lane] = zz;
      }
      __syncwarp();
      stg += (size_t)nb * STR;
    }
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  if (!ok) {
    if (lane == 0) atomicExch(err, 2);
    return;
  }
  // restricted prolongation (R_i^0)^T: owned rows only
  for (int idx = lane; idx < 7 * m; idx += 32) {
    const int q = idx / 7, cc = idx - 7 * q;
    if (R.owned[r0 + q]) z[7 * (int64_t)R.gnode[r0 + q] + cc] = (double)w[idx];
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
  return 128 + (size_t)NST * r.stage_blocks * Pack<TF>::stride * sizeof(TF) + (size_t)7 * r.max_rows * sizeof(TF);
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
cudaError_t launch_ras_apply_stream(const RasStreamDev& r, const double* rin, double* z, int32_t* err,
                                    cudaStream_t s) {
  const size_t sm = ras_stream_smem<TF>(r);
  cudaError_t e = cudaFuncSetAttribute(k_ras_apply_stream<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_ras_apply_stream<TF><<<r.np, 64, sm, s>>>(r, rin, z, err);
  return cudaGetLastError();
}

template size_t ras_stream_smem<float>(const RasStreamDev&);
template size_t ras_stream_smem<double>(const RasStreamDev&);
template void launch_pack_factors<float>(const RasStreamDev&, const float*, cudaStream_t);
template void launch_pack_factors<double>(const RasStreamDev&, const double*, cudaStream_t);
template cudaError_t launch_ras_apply_stream<float>(const RasStreamDev&, const double*, double*, int32_t*,
                                                    cudaStream_t);
template cudaError_t launch_ras_apply_stream<double>(const RasStreamDev&, const double*, double*, int32_t*,
                                                     cudaStream_t);

}  // namespace fsi
