// Test harness: exposes the solver's host-side Schwarz plan (csrc/setup.cpp) to
// the CPU tests through a small C interface, so that the partition, overlap,
// subdomain orderings and ILU(k) fill patterns can be compared with the oracle
// without a GPU. Built by tests/test_host_plan.py with the host compiler.
#include <cstring>
#include <string>
#include <vector>

#include "setup.h"

using namespace fsi;

struct PlanBox {
  BsrPattern P;
  RasPlan R;
};

extern "C" void* plan_new(int64_t n, const double* X, int64_t T, const int32_t* tets, const int32_t* node_problem,
                          int32_t n_problems, int32_t np, int32_t overlap, int32_t fill, int32_t ordering,
                          const uint8_t* rank) {
  auto* b = new PlanBox;
  std::vector<int32_t> tv(tets, tets + 4 * T);
  b->P = build_pattern(n, tv);
  b->R = build_ras(b->P, X, n, node_problem, n_problems, np, overlap, fill, ordering, rank);
  return b;
}

extern "C" void plan_free(void* p) { delete static_cast<PlanBox*>(p); }

// data pointer and element count of a named plan array (elements are int64
// unless noted: gnode, col, sd_depth int32; owned uint8)
extern "C" const void* plan_array(void* p, const char* name, int64_t* count) {
  RasPlan& R = static_cast<PlanBox*>(p)->R;
  const std::string s(name);
#define ARR(field)                        \
  if (s == #field) {                      \
    *count = (int64_t)R.field.size();     \
    return R.field.data();                \
  }
  ARR(sd_row) ARR(gnode) ARR(owned) ARR(row_ptr) ARR(col) ARR(diag) ARR(sd_depth) ARR(sd_item) ARR(item_row)
#undef ARR
  *count = -1;
  return nullptr;
}
