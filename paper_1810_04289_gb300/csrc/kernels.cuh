// Launch wrappers of the solver's CUDA kernels (definitions in assembly.cu,
// sparse.cu, krylov.cu). All take raw device pointers and a stream.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "element.cuh"

namespace fsi {

// per-problem inflow data: center[3], normal[3], radius, peak, amp, freq, phase
constexpr int INLET_STRIDE = 11;

struct MeshDev {
  int64_t N, T, Tf;          // nodes, tets, fluid tets (tets [0, Tf) fluid, [Tf, T) wall)
  const double* X;           // [N*3]
  const int32_t* tets;       // [T*4]
  const uint32_t* nflag;     // [N]
  const int32_t* nprob;      // [N]
  const double* inlet;       // [nprob*INLET_STRIDE]
};

// ---- wall shear stress (wss.cu): face = 4 * fluid tet + local index of the
// vertex opposite the face; fb = [P+1] face offsets of the problems
void launch_wss(const MeshDev& m, double mu, int64_t nf, const int64_t* face, const int64_t* fb, int32_t P,
                const double* y, double* wss, double* marea, double* area, double* sawss, cudaStream_t s);

// ---- assembly (assembly.cu)
void launch_elem_residual(const MeshDev& m, const MatConst& mc, const double* y, const double* y1,
                          const double* y2, double* Fe, cudaStream_t s);
void launch_gather_residual(const MeshDev& m, const int64_t* nptr, const int32_t* nsrc, const double* Fe,
                            double* F, cudaStream_t s);
void launch_constraint_residual(const MeshDev& m, const MatConst& mc, double t, const double* y,
                                const double* y1, double* F, cudaStream_t s);
// Xl: per-tet reference coordinates relative to vertex 0 (12 per tet); y, y1, y2
// node states, all in the arithmetic type T
// element Jacobians of the tets [t0, t1) into Ke (784 values per tet, from tet t0)
template <class T>
void launch_elem_jacobian(const MeshDev& m, const MatConst& mc, const T* Xl, const T* y, const T* y1, const T* y2,
                          T* Ke, int64_t t0, int64_t t1, cudaStream_t s);
// out = [a | b | c] converted to FP32 (3 n floats)
void launch_states_to_float(int64_t n, const double* a, const double* b, const double* c, float* out,
                            cudaStream_t s);
// add the element blocks of the tets [t0, t1) (Ke as above) into the BSR values;
// t0 = 0 starts the sums
template <class T>
void launch_gather_jacobian(int64_t nnzb, const int64_t* bptr, const int32_t* bsrc, const T* Ke, T* vals,
                            int64_t t0, int64_t t1, cudaStream_t s);
template <class T>
void launch_constraint_jacobian(const MeshDev& m, const MatConst& mc, const int32_t* diag, T* vals,
                                cudaStream_t s);

// ---- sparse (sparse.cu)
// y = J x; threads_per_row 32 (one warp per block row) or 16 (two rows per
// warp); guard: optional device flag, the kernel does nothing while *guard == 0
template <class TV, class TX>
void launch_bsr_spmv(int64_t n, const int64_t* row_ptr, const int32_t* col, const TV* vals, const TX* x,
                     double* y, int threads_per_row, const int* guard, cudaStream_t s);
void launch_to_float(int64_t n, const double* x, float* y, const int* guard, cudaStream_t s);

struct RasDev {
  int32_t np;
  const int64_t* sd_row;
  const int32_t* gnode;
  const uint8_t* owned;
  const int64_t* row_ptr;
  const int32_t* col;
  const int64_t* gblk;
  const int64_t* diag;
  const int64_t* lent_ptr;
  const int64_t* lent_pos;
  const int64_t* lent_kdiag;
  const int64_t* upd_ptr;
  const int64_t* upd_tgt;
  const int64_t* upd_src;
  const int64_t* sd_lvlL;
  const int64_t* sd_lvlU;
  const int64_t* lvlL_ptr;
  const int64_t* lvlU_ptr;
  const int32_t* lvlL_rows;
  const int32_t* lvlU_rows;
  int64_t nblocks;
  int32_t max_row_blocks;  // most blocks in one factor row
  int32_t max_row_lent;    // most L blocks in one row
  int32_t max_row_upd;     // most elimination updates in one row
  int32_t max_entry_upd;   // most updates of one L block
  int32_t factor_mode;     // factorisation kernel: 0..2 rows in order (shared-memory modes), 3 nested-dissection groups
  const int32_t* sd_depth; // [np] nested-dissection depth of each subdomain (0: one item)
  const int64_t* sd_item;  // [np+1] first item of each subdomain
  const int64_t* item_row; // [items] end row of each item (subdomain-relative)
  int32_t max_depth;       // deepest dissection (the nested-dissection factorisation uses 2^max_depth groups)
};
template <class TF, class TJ>
void launch_ras_extract(const RasDev& r, const TJ* vals, TF* fac, cudaStream_t s);
template <class TF>
void launch_ras_factor(const RasDev& r, TF* fac, int32_t* err, cudaStream_t s);
template <class TF>
bool ras_factor_fits(const RasDev& r, int mode);  // mode 0..3 fits one CTA
// shared-memory limit of the factorisation CTA (the opt-in maximum)
constexpr size_t FACTOR_SMEM_MAX = 227 * 1024;
template <class TF>
void launch_ras_apply(const RasDev& r, const TF* fac, const double* rin, TF* work, double* z, float* z32,
                      const int* guard, cudaStream_t s);

// ---- streamed RAS apply (ras_stream.cu)
struct RasStreamDev {
  int32_t np;
  const int64_t* sd_row;
  const int32_t* gnode;
  const uint8_t* owned;
  const int64_t* L_cnt;   // [rows] L blocks of each row
  const int64_t* U_cnt;   // [rows] 1 (inverted pivot) + U blocks of each row
  const int64_t* L_off;   // [np+1] first packed L block of each subdomain
  const int64_t* U_off;   // [np+1] first packed U block of each subdomain
  void* Lpack;
  void* Upack;
  int64_t nL, nU;
  const int64_t* Lsrc;    // [nL] factor block copied into each packed L block
  const int32_t* Lcol;    // [nL] subdomain-relative column row
  const int64_t* Usrc;
  const int32_t* Ucol;
  const int64_t* Upiv;    // [nU] factor block of the row's inverted pivot, -1 for the pivot itself
  int32_t stage_blocks;   // blocks per ring stage (one bulk copy; rows may straddle stages)
  int64_t max_rows;       // rows of the largest subdomain
  int32_t nst;            // ring stages in flight per warp (2..8)
  int32_t stall;          // tests only: the producer issues nothing (bounded waits run out)
  // nested-dissection items (one item per subdomain for the other orderings)
  const int32_t* sd_depth;  // [np] depth D: 2^(D+1) - 1 items, solved by 2^D warps
  const int64_t* sd_item;   // [np+1] first item of each subdomain
  const int64_t* item_row;  // [items] end row of each item (subdomain-relative)
  const int32_t* item_blk;  // [items][4] first / end block of the item in the subdomain's L and U streams
  int32_t max_depth;        // deepest D (the CTA has 2^max_depth warps)
};
template <class TF>
size_t ras_stream_smem(const RasStreamDev& r);
template <class TF>
void launch_pack_factors(const RasStreamDev& r, const TF* fac, cudaStream_t s);
// once per context: allow the apply kernel its dynamic shared memory
template <class TF>
cudaError_t ras_stream_init(const RasStreamDev& r);
// z = B^{-1} r; z32 (optional) receives an FP32 copy; guard as for the SpMV
template <class TF>
cudaError_t launch_ras_apply_stream(const RasStreamDev& r, const double* rin, double* z, float* z32, int32_t* err,
                                    const int* guard, cudaStream_t s);

// ---- batched Krylov / BLAS-1 (krylov.cu): vectors of n doubles holding P
// independent problems one after the other; reductions are segmented by
// problem over a fixed chunk table (deterministic). guard: optional device
// flag; guarded kernels do nothing while *guard == 0.
struct SegDev {
  int32_t P;                 // problems
  int64_t n_chunks;
  const int64_t* chunk_beg;  // [n_chunks+1] first dof of each chunk (chunks never straddle problems)
  const int64_t* prob_chunk; // [P+1] chunks of each problem
  const int32_t* node_prob;  // [N] problem of each node
  int* counter;              // [P * SEG_GROUPS] blocks done per (problem, vector group); zero between launches
};
constexpr int SEG_GROUPS = 9;  // vector groups of 8 in one multi-dot (restart <= 64 -> at most 65 vectors)
// out[p * ldo + k] = V_k . w for k < nv (and, with_self, out[p * ldo + nv] = w . w);
// returns the number of kernels launched (1 or 2)
int launch_seg_mdot(const SegDev& sg, int32_t nv, const double* V, int64_t ldv, const double* w, double* partial,
                    double* out, int32_t ldo, const int* guard, cudaStream_t s, int with_self = 0);
// selective reorthogonalisation test after one Gram-Schmidt pass (see krylov.cu)
void launch_seg_reorth_decide(int32_t P, const double* ws, const double* nrm, int32_t ldn, double* hb, int32_t lda,
                              int32_t j, const int* active, int* flag, cudaStream_t s);
void launch_seg_norm(const SegDev& sg, const double* x, double* partial, double* out, int32_t ldo,
                     const int* guard, cudaStream_t s);
// w -= V h per problem, then w *= scal[p] (scal optional)
void launch_seg_maxpy(const SegDev& sg, int64_t n, int32_t nv, const double* V, int64_t ldv, const double* h,
                      int32_t ldh, double* w, const int* guard, cudaStream_t s, const double* scal = nullptr);
// the new Arnoldi vector's norm as sqrt(||w||^2 - ||h2||^2) where that is safe (see krylov.cu)
void launch_seg_norm_pythagoras(int32_t P, const double* hb, int32_t lda, int32_t j, double* hsub, int64_t ldsub,
                                double* inv, int* unsafe, int* flag, int force, const int* guard, cudaStream_t s);
void launch_seg_norm_fix(int32_t P, const double* nrm, const int* unsafe, double* hsub, int64_t ldsub, double* scal,
                         const int* guard, cudaStream_t s);
void launch_seg_scale_inv(const SegDev& sg, int64_t n, const double* x, const double* scal, int32_t lds,
                          double* y, const int* guard, cudaStream_t s);

void launch_seg_cycle_init(int32_t P, double* g, int32_t ldg, const double* beta, const double* target, int* active,
                           int* kcols, int* any, cudaStream_t s);
// column j of each active problem's Hessenberg = a + b (the two Gram-Schmidt passes, lda apart per
// problem), then the Givens update
void launch_seg_givens(int32_t P, const double* a, const double* b, int32_t lda, double* H, int32_t ldh, int32_t m,
                       int32_t j, double* cs, double* sn, double* g, double* res, const double* target, int* active,
                       int* kcols, int* any, cudaStream_t s);
void launch_seg_lsq(int32_t P, const double* H, int32_t ldh, int32_t m, const int* kcols, const double* g, double* y,
                    cudaStream_t s);
void launch_seg_update_x(const SegDev& sg, int64_t n, const double* Z, int64_t ldz, const double* y, int32_t m,
                         const int* kcols, double* x, cudaStream_t s);
void launch_seg_axpy(const SegDev& sg, int64_t n, const double* x, const double* alpha, const double* y, double* out,
                     cudaStream_t s);
void launch_seg_neg_masked(const SegDev& sg, int64_t n, const double* x, const int* mask, double* out,
                           cudaStream_t s);
void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s);
void launch_copy(int64_t n, const double* x, double* y, cudaStream_t s);
void launch_fill(int64_t n, double v, double* x, cudaStream_t s);

}  // namespace fsi
