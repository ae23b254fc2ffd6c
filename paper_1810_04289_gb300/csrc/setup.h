// Host-side symbolic setup of the solver: block-sparse pattern, assembly gather
// lists, Schwarz subdomains (partition, overlap, RCM order), ILU(k) update lists
// and level schedules. Everything here runs once per mesh in fsi_create.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fsi {

// node flags (device-side row routing and constraint rows)
enum : uint32_t {
  NF_U_KIN = 1,      // u rows: u - (d - d_old)/dt (interface, Eq. 3 kinematic condition)
  NF_U_IDENT = 2,    // u rows: u = 0 (wall-only node)
  NF_P_IDENT = 4,    // p row: p = 0 (wall-only node)
  NF_U_INLET = 8,    // u rows: u = inflow profile (Eq. 3 inlet)
  NF_D_ZERO = 16,    // d rows: d = 0 (caps: Eq. 1 d_m = 0, Eq. 2 clamped wall end)
  NF_ITF = 32,       // interface node: fluid momentum goes to the d rows
  NF_FLUID = 64,
  NF_U_CONSTR = NF_U_KIN | NF_U_IDENT | NF_U_INLET
};

struct BsrPattern {
  int64_t n = 0;                 // block rows
  std::vector<int64_t> row_ptr;  // [n+1]
  std::vector<int32_t> col;      // [nnzb], sorted per row
  std::vector<int32_t> diag;     // [n] position of the diagonal block
};

// Pattern = node adjacency through tets, plus the diagonal.
BsrPattern build_pattern(int64_t n_nodes, const std::vector<int32_t>& tets);

// Gather lists of the atomic-free assembly: for every block (resp. node) the
// element-buffer slots that add into it, in increasing tet order.
//   block k: sum over c in [bptr[k], bptr[k+1]) of Ke sub-block bsrc[c]
//            (bsrc = tet*16 + a*4 + b)
//   node i : sum over c in [nptr[i], nptr[i+1]) of Fe row block nsrc[c]
//            (nsrc = tet*4 + a)
void build_gather(const BsrPattern& P, const std::vector<int32_t>& tets,
                  std::vector<int64_t>& bptr, std::vector<int32_t>& bsrc,
                  std::vector<int64_t>& nptr, std::vector<int32_t>& nsrc);

// Restricted additive Schwarz plan (Eq. 14-16), concatenated over subdomains.
struct RasPlan {
  int32_t np = 0;
  std::vector<int64_t> sd_row;     // [np+1] local-row offsets
  std::vector<int32_t> gnode;      // [rows] global node of each local row (RCM order)
  std::vector<uint8_t> owned;      // [rows] 1 if the node belongs to the subdomain (R_i^0)
  std::vector<int64_t> row_ptr;    // [rows+1] into the block arrays
  std::vector<int32_t> col;        // [blocks] column as a concatenated local row index
  std::vector<int64_t> gblk;       // [blocks] global BSR block extracted into it, -1 = fill
  std::vector<int64_t> diag;       // [rows] position of the diagonal block
  // ILU elimination lists: for each row, its L blocks in column order; for each
  // L block (i,k), the updates A_ij -= A_ik A_kj with (i,j) in the pattern
  std::vector<int64_t> lent_ptr;   // [rows+1]
  std::vector<int64_t> lent_pos;   // [nL] position of A_ik
  std::vector<int64_t> lent_kdiag; // [nL] position of A_kk (inverted pivot)
  std::vector<int64_t> upd_ptr;    // [nL+1]
  std::vector<int64_t> upd_tgt;    // [nU] position of A_ij
  std::vector<int64_t> upd_src;    // [nU] position of A_kj
  // level schedules (rows of one level are independent)
  std::vector<int64_t> sd_lvlL, sd_lvlU;     // [np+1] offsets into the level arrays
  std::vector<int64_t> lvlL_ptr, lvlU_ptr;   // [levels+1] into lvl*_rows
  std::vector<int32_t> lvlL_rows, lvlU_rows; // concatenated local rows (subdomain-relative)
  int32_t max_levels = 0;
  int64_t max_rows = 0;
  // nested-dissection items of each subdomain (one item, depth 0, for the
  // other orderings): 2^(D+1) - 1 items in phase-major order (the 2^D leaves,
  // then the separators from the deepest level up to the root's); item k of
  // subdomain s ends at local row item_row[sd_item[s] + k] (item 0 starts at 0)
  std::vector<int32_t> sd_depth;   // [np] D
  std::vector<int64_t> sd_item;    // [np+1]
  std::vector<int64_t> item_row;   // [sum of items]
  int32_t max_depth = 0;
};

// smallest average leaf of the nested-dissection ordering: the depth D of a
// subdomain of m rows is the largest D <= 3 with m >= ND_MIN_LEAF * 2^D
constexpr int32_t ND_MIN_LEAF = 48;

// fill_level k: pattern of the level-of-fill ILU(k) of each J_i^delta (0 = the
// pattern of J_i^delta itself). ordering of each subdomain: 0 natural (global
// node order), 1 reverse Cuthill-McKee, 2 reverse Cuthill-McKee stably sorted
// by node_rank (lumen nodes 0, interface 1, wall 2), 3 nested dissection
// (coordinate bisection, one-sided vertex separators) with reverse
// Cuthill-McKee inside every part.
RasPlan build_ras(const BsrPattern& P, const double* X, int64_t n_nodes, const int32_t* node_problem,
                  int32_t n_problems, int32_t np, int32_t overlap, int32_t fill_level, int32_t ordering,
                  const uint8_t* node_rank);

}  // namespace fsi
