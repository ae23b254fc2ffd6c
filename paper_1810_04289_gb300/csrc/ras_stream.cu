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
//   U stream: for every row in decreasing order, its inverted pivot D_q^{-1}, then
//             its U blocks premultiplied and negated, -D_q^{-1} U_qj.
// Each packed block holds its 7 rows as 8-wide, 16-byte aligned rows (56 values):
// the row's 7 entries, then one slot; row 0's slot holds the subdomain-relative
// column row (as int bits). The subdomain vector in shared memory is 8 wide too,
// so each 7-term product is four 16-byte loads (FP32) instead of fourteen.
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
// packed block: 7 rows of 8 values (the 7 entries of the row, then one slot),
// 16-byte aligned rows; the slot of row 0 holds the column (as int bits), the
// other slots are zero
template <class TF> struct Pack { static constexpr int stride = 56; };

template <class TF>
__device__ __forceinline__ int blk_col(const TF* blk) {
  return *reinterpret_cast<const int*>(blk + 7);
}

// the 7-term product of row c of a packed block with the node vector x (8 wide):
// 16-byte loads of the row and of x
__device__ __forceinline__ float row7(const float* a, const float* x) {
  const float4 a0 = *reinterpret_cast<const float4*>(a), a1 = *reinterpret_cast<const float4*>(a + 4);
  const float4 x0 = *reinterpret_cast<const float4*>(x), x1 = *reinterpret_cast<const float4*>(x + 4);
  const float p01 = a0.x * x0.x + a0.y * x0.y;
  const float p23 = a0.z * x0.z + a0.w * x0.w;
  const float p45 = a1.x * x1.x + a1.y * x1.y;
  return (p01 + p23) + (p45 + a1.z * x1.z);
}
__device__ __forceinline__ double row7(const double* a, const double* x) {
  const double2 a0 = *reinterpret_cast<const double2*>(a), a1 = *reinterpret_cast<const double2*>(a + 2);
  const double2 a2 = *reinterpret_cast<const double2*>(a + 4), a3 = *reinterpret_cast<const double2*>(a + 6);
  const double2 x0 = *reinterpret_cast<const double2*>(x), x1 = *reinterpret_cast<const double2*>(x + 2);
  const double2 x2 = *reinterpret_cast<const double2*>(x + 4), x3 = *reinterpret_cast<const double2*>(x + 6);
  const double p01 = a0.x * x0.x + a0.y * x0.y;
  const double p23 = a1.x * x1.x + a1.y * x1.y;
  const double p45 = a2.x * x2.x + a2.y * x2.y;
  return (p01 + p23) + (p45 + a3.x * x3.x);
}

constexpr int NSTMAX = 8;  // most ring stages (runtime count R.nst)

// sum over blocks b in [0, nb) of (block b, row c) . w[col(b)], reduced over
// the warp: lane = 7 j + c handles blocks j, j + 4, ...; every block
// gathers its column index first so that all loads of a chunk are independent,
// then forms the 7-term products (16-byte loads of the block row and of the
// 8-wide node vector). The total lands in lanes 0..6.
template <class TF, int STR>
__device__ __forceinline__ TF row_dot(const TF* stg, int nb, const TF* w, int j, int c) {
  TF acc = TF(0);
  if (j < 4) {
    // 32-bit element offsets within the stage (a stage fits in shared memory)
    for (int b = j; b < nb; b += 16) {
      int cols[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int bi = b + 4 * i;
        cols[i] = bi < nb ? blk_col(stg + bi * STR) : -1;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (cols[i] >= 0) acc += row7(stg + (b + 4 * i) * STR + 8 * c, w + 8 * cols[i]);
      }
    }
  }
  acc += __shfl_down_sync(0xffffffffu, acc, 14);
  acc += __shfl_down_sync(0xffffffffu, acc, 7);
  return acc;
}

// One warp's stream of factor stages. The warp walks, in order, the segments of
// the items it solves: forward phases 0..D (its item's L blocks), then backward
// phases D..0 (its item's U blocks). Lane 0 keeps NST bulk copies in flight
// along that sequence, into the warp's own ring, across phase boundaries (the
// factor bytes do not depend on the solve, so the next phase's first stages
// arrive while the CTA waits at the phase barrier).
struct WarpFeed {
  int D, wi;         // nested-dissection depth of the subdomain, warp index
  int seg;           // producer: current segment 0 .. 2D+1 (2D+2 = done)
  int pos, end;      // producer: next block to issue and end block of the current segment
  int issued, used;  // stages issued / consumed by this warp
  int islot;         // producer: ring slot of the next issue (issued mod NST)
  int uslot, uphase; // consumer: ring slot of the next stage (used mod NST) and its mbarrier phase parity
};

// item of segment j for warp wi, or -1 when the warp has no item in that phase
__device__ __forceinline__ int seg_item(int D, int wi, int j) {
  const int p = j <= D ? j : 2 * D + 1 - j;
  if (wi >= (1 << (D - p))) return -1;
  return (1 << (D + 1)) - (1 << (D - p + 1)) + wi;
}

// lane 0: move the producer to the first segment at or after f.seg that has
// blocks left, loading its bounds once (segment changes are rare: 2D + 2 per apply)
__device__ __forceinline__ void feed_seek(WarpFeed& f, const int32_t* ib) {
  while (f.pos >= f.end && f.seg <= 2 * f.D + 1) {
    if (++f.seg > 2 * f.D + 1) break;
    const int it = seg_item(f.D, f.wi, f.seg);
    if (it >= 0) {
      const bool isL = f.seg <= f.D;
      f.pos = ib[4 * it + (isL ? 0 : 2)];
      f.end = ib[4 * it + (isL ? 1 : 3)];
    }
  }
}

// lane 0: issue the next stage of the warp's sequence (if any) into its ring slot.
// The slot was last read by this warp's lanes, whose loads completed before the
// __syncwarp that precedes every call.
template <class TF, int STR>
__device__ __forceinline__ void feed_issue(WarpFeed& f, const int32_t* ib, const TF* Lpack, const TF* Upack, TF* ring,
                                           uint64_t* full, int NST, int SB) {
  feed_seek(f, ib);
  if (f.pos >= f.end) return;
  const int nb = min(SB, f.end - f.pos);
  const int st = f.islot;
  const uint32_t bytes = (uint32_t)(nb * STR * sizeof(TF));
  mbar_arrive_expect_tx(&full[st], bytes);
  bulk_g2s(ring + (size_t)st * SB * STR, (f.seg <= f.D ? Lpack : Upack) + (size_t)f.pos * STR, bytes, &full[st]);
  f.pos += nb;
  f.issued++;
  if (++f.islot == NST) f.islot = 0;
}

// Multi-warp streamed RAS apply (Sec. 3, Eq. 16) on nested-dissection ordered
// subdomains (Sec. 4.5): one CTA per subdomain; in each phase of the forward
// solve (leaves, then the separators level by level up to the root's) every item
// of the phase is solved by its own warp, the items of a phase being independent
// (no edge and no fill between them); the backward solve runs the phases in
// reverse. Subdomains in the other orderings are one item (depth 0): one warp.
// Each warp is its own producer: lane 0 streams the packed factor blocks of the
// warp's items through a ring of NST stages of SB blocks (cp.async.bulk with
// mbarrier completion); the warp solves the rows of the current stage (rows may
// straddle stages) on the subdomain vector in shared memory.
template <class TF>
__global__ void __launch_bounds__(256) k_ras_apply_stream(RasStreamDev R, const double* __restrict__ rin,
                                                          double* __restrict__ z, float* __restrict__ z32,
                                                          int32_t* err, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  constexpr int STR = Pack<TF>::stride;
  extern __shared__ __align__(128) unsigned char smem[];
  const int NST = R.nst;
  const int SB = R.stage_blocks;
  const int nwarps = blockDim.x >> 5;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);                     // [nwarps][NSTMAX]
  TF* rings = reinterpret_cast<TF*>(smem + 128 * ((nwarps * NSTMAX * 8 + 127) / 128));
  TF* ring = rings + (size_t)wi * NST * SB * STR;
  TF* w = rings + (size_t)nwarps * NST * SB * STR;
  unsigned short* Lcnt = reinterpret_cast<unsigned short*>(w + 8 * (size_t)R.max_rows);
  unsigned short* Ucnt = Lcnt + R.max_rows;
  uint64_t* full = bars + wi * NSTMAX;
  const int s = blockIdx.x;
  const int64_t r0 = R.sd_row[s];
  const int m = (int)(R.sd_row[s + 1] - r0);
  const int D = R.sd_depth[s];
  const int32_t* ib = R.item_blk + 4 * R.sd_item[s];        // per item: L begin, L end, U begin, U end
  const int64_t* irow = R.item_row + R.sd_item[s];          // per item: end row
  const TF* Lpack = reinterpret_cast<const TF*>(R.Lpack) + (size_t)R.L_off[s] * STR;
  const TF* Upack = reinterpret_cast<const TF*>(R.Upack) + (size_t)R.U_off[s] * STR;

  if (lane == 0)
    for (int i = 0; i < NST; ++i) mbar_init(&full[i], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // restriction R_i^delta r into shared memory
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const double* src = rin + 7 * (int64_t)R.gnode[r0 + q];
    double v[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) v[c] = src[c];
#pragma unroll
    for (int c = 0; c < 7; ++c) w[8 * q + c] = (TF)v[c];
    w[8 * q + 7] = TF(0);
    Lcnt[q] = (unsigned short)R.L_cnt[r0 + q];
    Ucnt[q] = (unsigned short)R.U_cnt[r0 + q];
  }
  __syncthreads();

  WarpFeed f{D, wi, -1, 0, 0, 0, 0, 0, 0, 0};
  const bool active = wi < (1 << D);
  if (active && lane == 0 && !R.stall)
    for (int k = 0; k < NST; ++k) feed_issue<TF, STR>(f, ib, Lpack, Upack, ring, full, NST, SB);
  f.issued = __shfl_sync(0xffffffffu, f.issued, 0);

  const int j = lane / 7, c = lane - 7 * (lane / 7);  // block slot 0..3 (4 = idle), component
  bool ok = true;
  // wait for the next stage of this warp's sequence; false on timeout
  auto next_stage = [&]() -> const TF* {
    const int st = f.uslot;
    if (!mbar_wait(&full[st], (uint32_t)f.uphase)) return nullptr;
    return ring + (size_t)st * SB * STR;
  };
  // the stage is consumed: lane 0 refills its slot with the next stage in line
  auto release = [&]() {
    __syncwarp();
    f.used++;
    if (++f.uslot == NST) {
      f.uslot = 0;
      f.uphase ^= 1;
    }
    if (lane == 0 && !R.stall) feed_issue<TF, STR>(f, ib, Lpack, Upack, ring, full, NST, SB);
    f.issued = __shfl_sync(0xffffffffu, f.issued, 0);
  };

  // forward: phases 0..D, w_q -= sum_k L_qk w_k over the rows of the warp's item
  for (int p = 0; p <= D; ++p) {
    const int it = seg_item(D, wi, p);
    if (it >= 0 && ok) {
      int q = it == 0 ? 0 : (int)irow[it - 1];
      const int qe = (int)irow[it];
      const int nLb = ib[4 * it + 1] - ib[4 * it];
      int rem = 0, done = 0;
      TF acc = TF(0);
      while (done < nLb) {
        const TF* stg = next_stage();
        if (!stg) { ok = false; break; }
        const int cap = min(SB, nLb - done);
        int pos = 0;
        if (rem > 0) {
          const int k = min(rem, cap);
          acc += row_dot<TF, STR>(stg, k, w, j, c);
          pos = k;
          rem -= k;
          if (rem == 0) {
            if (lane < 7) w[8 * q + lane] -= acc;
            __syncwarp();
            ++q;
          }
        }
        if (rem == 0) {
          for (; q < qe; ++q) {
            const int nb = Lcnt[q];
            if (pos + nb > cap) break;
            const TF a = row_dot<TF, STR>(stg + pos * STR, nb, w, j, c);
            if (lane < 7 && nb > 0) w[8 * q + lane] -= a;
            __syncwarp();
            pos += nb;
          }
          if (q < qe && pos < cap) {
            acc = row_dot<TF, STR>(stg + pos * STR, cap - pos, w, j, c);
            rem = Lcnt[q] - (cap - pos);
          }
        }
        done += cap;
        release();
      }
    }
    __syncthreads();
  }
  // backward: phases D..0, w_q = D_q^{-1} w_q - sum_j (D_q^{-1} U_qj) w_j: the
  // U stream holds, per row, the inverted pivot (column q: it multiplies the
  // forward result still in w_q) and then the blocks -D_q^{-1} U_qj, so a row is
  // one dot product over its blocks, as in the forward solve
  for (int p = D; p >= 0; --p) {
    const int it = seg_item(D, wi, 2 * D + 1 - p);
    if (it >= 0 && ok) {
      const int qb = it == 0 ? 0 : (int)irow[it - 1];
      int q = (int)irow[it] - 1;
      const int nUb = ib[4 * it + 3] - ib[4 * it + 2];
      int rem = 0, done = 0;
      TF acc = TF(0);
      while (done < nUb) {
        const TF* stg = next_stage();
        if (!stg) { ok = false; break; }
        const int cap = min(SB, nUb - done);
        int pos = 0;
        if (rem > 0) {
          const int k = min(rem, cap);
          acc += row_dot<TF, STR>(stg, k, w, j, c);
          pos = k;
          rem -= k;
          if (rem == 0) {
            if (lane < 7) w[8 * q + lane] = acc;
            __syncwarp();
            --q;
          }
        }
        if (rem == 0) {
          for (; q >= qb; --q) {
            const int nb = Ucnt[q];
            if (pos + nb > cap) break;
            const TF a = row_dot<TF, STR>(stg + pos * STR, nb, w, j, c);
            if (lane < 7) w[8 * q + lane] = a;
            __syncwarp();
            pos += nb;
          }
          if (q >= qb && pos < cap) {
            acc = row_dot<TF, STR>(stg + pos * STR, cap - pos, w, j, c);
            rem = Ucnt[q] - (cap - pos);
          }
        }
        done += cap;
        release();
      }
    }
    __syncthreads();
  }
  if (!ok) {
    // a wait gave up: record it and let this warp's copies still in flight land
    // (bounded) before the CTA exits
    if (lane == 0) {
      atomicExch(err, 2);
      for (int k = f.used; k < f.issued; ++k) mbar_wait(&full[k % NST], (k / NST) & 1);
    }
  }
  __syncthreads();
  // restricted prolongation (R_i^0)^T: owned rows only
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    if (R.owned[r0 + q]) {
      const int64_t g7 = 7 * (int64_t)R.gnode[r0 + q];
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) z[g7 + cc] = (double)w[8 * q + cc];
      if (z32) {
#pragma unroll
        for (int cc = 0; cc < 7; ++cc) z32[g7 + cc] = (float)w[8 * q + cc];
      }
    }
  }
}

// copy the factor blocks into the packed streams (7 rows of 8: the row's 7
// entries, then the column index in row 0's last slot, zeros in the others); a
// U block with a pivot (Upiv >= 0) is stored as -D_q^{-1} U_qj, the row's
// inverted pivot itself as it is
template <class TF>
__global__ void k_pack_factors(int64_t nL, const int64_t* __restrict__ Lsrc, const int32_t* __restrict__ Lcol,
                               int64_t nU, const int64_t* __restrict__ Usrc, const int32_t* __restrict__ Ucol,
                               const int64_t* __restrict__ Upiv, const TF* __restrict__ fac, TF* __restrict__ Lpack,
                               TF* __restrict__ Upack) {
  constexpr int STR = Pack<TF>::stride;
  const int64_t total = (nL + nU) * STR;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / STR;
    const int e = (int)(idx - STR * b);
    const int r = e >> 3, k = e & 7;
    const bool isL = b < nL;
    const int64_t bb = isL ? b : b - nL;
    const int64_t src = isL ? Lsrc[bb] : Usrc[bb];
    TF* dst = (isL ? Lpack : Upack) + bb * STR;
    if (k < 7) {
      const int64_t piv = isL ? -1 : Upiv[bb];
      if (piv < 0) {
        dst[e] = fac[49 * src + 7 * r + k];
      } else {
        // -(D_q^{-1} U_qj)[r][k]
        const TF* Dq = fac + 49 * piv + 7 * r;
        const TF* U = fac + 49 * src + k;
        TF v = TF(0);
#pragma unroll
        for (int mm = 0; mm < 7; ++mm) v += Dq[mm] * U[7 * mm];
        dst[e] = -v;
      }
    } else if (r == 0) {
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
  const size_t W = (size_t)1 << r.max_depth;
  return 128 * ((W * NSTMAX * 8 + 127) / 128) + W * r.nst * r.stage_blocks * Pack<TF>::stride * sizeof(TF) +
         (size_t)8 * r.max_rows * sizeof(TF) + (size_t)4 * r.max_rows + 16;
}

template <class TF>
void launch_pack_factors(const RasStreamDev& r, const TF* fac, cudaStream_t s) {
  const int64_t total = (r.nL + r.nU) * Pack<TF>::stride;
  int64_t g = (total + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_pack_factors<TF><<<(int)g, 256, 0, s>>>(r.nL, r.Lsrc, r.Lcol, r.nU, r.Usrc, r.Ucol, r.Upiv, fac,
                                            (TF*)r.Lpack, (TF*)r.Upack);
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
  k_ras_apply_stream<TF><<<r.np, 32 << r.max_depth, ras_stream_smem<TF>(r), s>>>(r, rin, z, z32, err, guard);
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
