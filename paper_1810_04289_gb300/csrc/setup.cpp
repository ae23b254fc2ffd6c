// Host-side symbolic setup (see setup.h).
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace fsi {

BsrPattern build_pattern(int64_t n, const std::vector<int32_t>& tets) {
  const int64_t T = (int64_t)tets.size() / 4;
  // count incident tets per node, gather neighbour candidates, sort-unique per row
  std::vector<int64_t> deg(n + 1, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a) deg[tets[4 * t + a] + 1] += 4;
  for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  std::vector<int32_t> cand(deg[n]);
  std::vector<int64_t> fill(deg.begin(), deg.end() - 1);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a) {
      int32_t i = tets[4 * t + a];
      for (int b = 0; b < 4; ++b) cand[fill[i]++] = tets[4 * t + b];
    }
  BsrPattern P;
  P.n = n;
  P.row_ptr.assign(n + 1, 0);
  P.diag.assign(n, -1);
  std::vector<int32_t> row;
  P.col.reserve(deg[n] / 3);
  for (int64_t i = 0; i < n; ++i) {
    row.assign(cand.begin() + deg[i], cand.begin() + deg[i + 1]);
    row.push_back((int32_t)i);
    std::sort(row.begin(), row.end());
    row.erase(std::unique(row.begin(), row.end()), row.end());
    for (int32_t j : row) {
      if (j == i) P.diag[i] = (int32_t)(P.col.size() - P.row_ptr[i]);
      P.col.push_back(j);
    }
    P.row_ptr[i + 1] = (int64_t)P.col.size();
  }
  for (int64_t i = 0; i < n; ++i) P.diag[i] = (int32_t)(P.row_ptr[i] + P.diag[i]);
  return P;
}

static inline int64_t find_block(const BsrPattern& P, int32_t i, int32_t j) {
  const int32_t* b = P.col.data() + P.row_ptr[i];
  const int32_t* e = P.col.data() + P.row_ptr[i + 1];
  const int32_t* it = std::lower_bound(b, e, j);
  if (it == e || *it != j) throw std::runtime_error("pattern lookup failed");
  return (int64_t)(it - P.col.data());
}

void build_gather(const BsrPattern& P, const std::vector<int32_t>& tets, std::vector<int64_t>& bptr,
                  std::vector<int32_t>& bsrc, std::vector<int64_t>& nptr, std::vector<int32_t>& nsrc) {
  const int64_t T = (int64_t)tets.size() / 4;
  const int64_t nnzb = (int64_t)P.col.size();
  std::vector<int64_t> blk(16 * T);
  bptr.assign(nnzb + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) blk[16 * t + 4 * a + b] = find_block(P, tets[4 * t + a], tets[4 * t + b]);
  for (int64_t q = 0; q < 16 * T; ++q) bptr[blk[q] + 1]++;
  for (int64_t k = 0; k < nnzb; ++k) bptr[k + 1] += bptr[k];
  bsrc.assign(16 * T, 0);
  std::vector<int64_t> f(bptr.begin(), bptr.end() - 1);
  for (int64_t t = 0; t < T; ++t)
    for (int s = 0; s < 16; ++s) bsrc[f[blk[16 * t + s]]++] = (int32_t)(16 * t + s);
  nptr.assign(P.n + 1, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a) nptr[tets[4 * t + a] + 1]++;
  for (int64_t i = 0; i < P.n; ++i) nptr[i + 1] += nptr[i];
  nsrc.assign(4 * T, 0);
  std::vector<int64_t> g(nptr.begin(), nptr.end() - 1);
  for (int64_t t = 0; t < T; ++t)
    for (int a = 0; a < 4; ++a) nsrc[g[tets[4 * t + a]]++] = (int32_t)(4 * t + a);
}

// ---------------------------------------------------------------------------
// Schwarz subdomains
// ---------------------------------------------------------------------------

// recursive coordinate bisection of `idx` into `parts` parts numbered from `first`
static void rcb(const double* X, std::vector<int32_t>& idx, int64_t lo, int64_t hi, int32_t parts,
                int32_t first, std::vector<int32_t>& owner) {
  if (parts <= 1 || hi - lo <= 1) {
    for (int64_t k = lo; k < hi; ++k) owner[idx[k]] = first;
    return;
  }
  double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
  for (int64_t k = lo; k < hi; ++k)
    for (int c = 0; c < 3; ++c) {
      bmin[c] = std::min(bmin[c], X[3 * (int64_t)idx[k] + c]);
      bmax[c] = std::max(bmax[c], X[3 * (int64_t)idx[k] + c]);
    }
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (bmax[c] - bmin[c] > bmax[ax] - bmin[ax]) ax = c;
  int32_t pl = parts / 2;
  int64_t mid = lo + (int64_t)((double)(hi - lo) * pl / parts);
  std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int32_t a, int32_t b) {
    double xa = X[3 * (int64_t)a + ax], xb = X[3 * (int64_t)b + ax];
    return xa < xb || (xa == xb && a < b);
  });
  rcb(X, idx, lo, mid, pl, first, owner);
  rcb(X, idx, mid, hi, parts - pl, first + pl, owner);
}

RasPlan build_ras(const BsrPattern& P, const double* X, int64_t n, const int32_t* node_problem,
                  int32_t n_problems, int32_t np_req, int32_t overlap, int32_t fill_level, int32_t ordering,
                  const uint8_t* node_rank) {
  RasPlan R;
  // 1. non-overlapping partition: subdomains shared out over the problems by
  //    node count, then recursive coordinate bisection inside each problem
  std::vector<std::vector<int32_t>> pnodes(n_problems);
  for (int64_t i = 0; i < n; ++i) pnodes[node_problem ? node_problem[i] : 0].push_back((int32_t)i);
  std::vector<int32_t> owner(n, -1);
  int32_t next = 0;
  for (int32_t p = 0; p < n_problems; ++p) {
    if (pnodes[p].empty()) continue;
    int32_t k = (int32_t)std::llround((double)np_req * (double)pnodes[p].size() / (double)n);
    k = std::max<int32_t>(1, std::min<int32_t>(k, (int32_t)pnodes[p].size()));
    rcb(X, pnodes[p], 0, (int64_t)pnodes[p].size(), k, next, owner);
    next += k;
  }
  const int32_t np = next;
  R.np = np;
  std::vector<std::vector<int32_t>> own(np);
  for (int64_t i = 0; i < n; ++i) own[owner[i]].push_back((int32_t)i);

  // 2-5 per subdomain, independent: each subdomain builds its own plan (local
  // positions) on one host thread, then the plans are concatenated in order
  auto init_plan = [](RasPlan& L) {
    L.sd_row.assign(1, 0);
    L.row_ptr.assign(1, 0);
    L.lent_ptr.assign(1, 0);
    L.upd_ptr.assign(1, 0);
    L.sd_lvlL.assign(1, 0);
    L.sd_lvlU.assign(1, 0);
    L.lvlL_ptr.assign(1, 0);
    L.lvlU_ptr.assign(1, 0);
    L.sd_item.assign(1, 0);
  };
  std::vector<RasPlan> subs(np);
#pragma omp parallel
  {
  std::vector<int32_t> loc(n, -1), mark(n, -1);
  // symbolic ILU(k) row in a sorted linked list over local columns (END = none),
  // with the level and the extraction source of each entry, and a dense map
  // from column to position for the update lists
  std::vector<int32_t> nxt(n + 1, -1), lev(n + 1, 0);
  std::vector<int64_t> src(n + 1, -1), posq(n + 1, -1);
#pragma omp for schedule(dynamic, 1)
  for (int32_t s = 0; s < np; ++s) {
    RasPlan& R = subs[s];
    init_plan(R);
    // 2. overlap: delta layers of graph neighbours (Sec. 3, Omega_i^delta)
    std::vector<int32_t> nodes = own[s];
    for (int32_t v : nodes) mark[v] = s;
    size_t frontier = 0;
    for (int32_t layer = 0; layer < overlap; ++layer) {
      size_t end = nodes.size();
      for (size_t q = frontier; q < end; ++q) {
        int32_t v = nodes[q];
        for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) {
          int32_t w = P.col[e];
          if (mark[w] != s) {
            mark[w] = s;
            nodes.push_back(w);
          }
        }
      }
      frontier = end;
    }
    const int64_t m = (int64_t)nodes.size();
    // 3. order of the overlapped subdomain: natural (global node order), reverse
    //    Cuthill-McKee, reverse Cuthill-McKee with lumen nodes before wall nodes,
    //    or nested dissection with reverse Cuthill-McKee inside each part
    for (int64_t q = 0; q < m; ++q) loc[nodes[q]] = (int32_t)q;
    std::vector<int32_t> order;
    order.reserve(m);
    // reverse Cuthill-McKee of the local nodes `mem` (the subgraph they induce:
    // part[w] == pid), appended to `order`: start at the unvisited node of least
    // degree (ties: lowest node number), move it to the last node a breadth-first
    // sweep reaches (neighbours in increasing node number), then number breadth
    // first with each node's new neighbours by (degree, node number); reversed
    std::vector<int32_t> part(m, 0), degl(m, 0);
    std::vector<uint8_t> seen(m, 0), s2(m, 0);
    auto rcm_part = [&](const std::vector<int32_t>& mem, int32_t pid) {
      for (int32_t q : mem) {
        int32_t v = nodes[q], d = 0;
        for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) {
          const int32_t w = loc[P.col[e]];
          if (w >= 0 && part[w] == pid && w != q) d++;
        }
        degl[q] = d;
        seen[q] = 0;
      }
      const size_t base = order.size();
      std::vector<int32_t> nb, bfs;
      size_t done = 0;
      while (done < mem.size()) {
        int32_t st = -1;
        for (int32_t q : mem)
          if (!seen[q] && (st < 0 || degl[q] < degl[st] || (degl[q] == degl[st] && nodes[q] < nodes[st]))) st = q;
        bfs.assign(1, st);
        s2[st] = 1;
        for (size_t h = 0; h < bfs.size(); ++h) {
          int32_t v = nodes[bfs[h]];
          for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) {
            int32_t w = loc[P.col[e]];
            if (w >= 0 && part[w] == pid && !s2[w] && !seen[w]) {
              s2[w] = 1;
              bfs.push_back(w);
            }
          }
        }
        for (int32_t q : bfs) s2[q] = 0;
        st = bfs.back();
        seen[st] = 1;
        size_t head = order.size();
        order.push_back(st);
        while (head < order.size()) {
          int32_t v = nodes[order[head++]];
          nb.clear();
          for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) {
            int32_t w = loc[P.col[e]];
            if (w >= 0 && part[w] == pid && !seen[w]) {
              seen[w] = 1;
              nb.push_back(w);
            }
          }
          std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
            return degl[a] < degl[b] || (degl[a] == degl[b] && nodes[a] < nodes[b]);
          });
          order.insert(order.end(), nb.begin(), nb.end());
        }
        done = order.size() - base;
      }
      std::reverse(order.begin() + base, order.end());
    };
    int32_t depth = 0;
    std::vector<int64_t> items{0};  // item row offsets (phase-major)
    if (ordering == 0) {
      for (int64_t q = 0; q < m; ++q) order.push_back((int32_t)q);
      std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return nodes[a] < nodes[b]; });
    } else if (ordering == 3) {
      // nested dissection of depth D (the largest D <= 3 with m / 2^D >= 48):
      // each piece is cut at the median of its longest coordinate axis (order
      // (coordinate, node number), lower half floor(n/2) nodes); the separator
      // is the lower half's nodes with a neighbour in the upper half. Items in
      // phase-major order: the 2^D leaves, then the separators from the deepest
      // level up to the root's; nodes within an item in reverse Cuthill-McKee order
      while (depth < 3 && m >= ((int64_t)ND_MIN_LEAF << (depth + 1))) ++depth;
      std::vector<std::vector<int32_t>> cur(1), next;
      for (int64_t q = 0; q < m; ++q) cur[0].push_back((int32_t)q);
      std::vector<std::vector<std::vector<int32_t>>> seps(depth);
      for (int32_t d = 0; d < depth; ++d) {
        next.clear();
        for (auto& S : cur) {
          double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
          for (int32_t q : S)
            for (int c = 0; c < 3; ++c) {
              bmin[c] = std::min(bmin[c], X[3 * (int64_t)nodes[q] + c]);
              bmax[c] = std::max(bmax[c], X[3 * (int64_t)nodes[q] + c]);
            }
          int ax = 0;
          for (int c = 1; c < 3; ++c)
            if (bmax[c] - bmin[c] > bmax[ax] - bmin[ax]) ax = c;
          std::sort(S.begin(), S.end(), [&](int32_t a, int32_t b) {
            const double xa = X[3 * (int64_t)nodes[a] + ax], xb = X[3 * (int64_t)nodes[b] + ax];
            return xa < xb || (xa == xb && nodes[a] < nodes[b]);
          });
          const size_t half = S.size() / 2;
          for (size_t k = 0; k < S.size(); ++k) part[S[k]] = k < half ? 1 : 2;
          std::vector<int32_t> A, B(S.begin() + half, S.end()), sep;
          for (size_t k = 0; k < half; ++k) {
            const int32_t q = S[k], v = nodes[q];
            bool cut = false;
            for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1] && !cut; ++e) {
              const int32_t w = loc[P.col[e]];
              cut = w >= 0 && part[w] == 2;
            }
            (cut ? sep : A).push_back(q);
          }
          for (int32_t q : S) part[q] = 0;
          next.push_back(std::move(A));
          next.push_back(std::move(B));
          seps[d].push_back(std::move(sep));
        }
        cur.swap(next);
      }
      // phase-major items, each ordered by RCM on the subgraph it induces
      std::vector<std::vector<int32_t>*> it;
      for (auto& S : cur) it.push_back(&S);
      for (int32_t d = depth - 1; d >= 0; --d)
        for (auto& S : seps[d]) it.push_back(&S);
      for (size_t k = 0; k < it.size(); ++k)
        for (int32_t q : *it[k]) part[q] = (int32_t)k + 1;
      for (size_t k = 0; k < it.size(); ++k) {
        rcm_part(*it[k], (int32_t)k + 1);
        items.push_back((int64_t)order.size());
      }
      for (int64_t q = 0; q < m; ++q) part[q] = 0;
    } else {
      std::vector<int32_t> all(m);
      for (int64_t q = 0; q < m; ++q) all[q] = (int32_t)q;
      rcm_part(all, 0);
      if (ordering == 2 && node_rank) {
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return node_rank[nodes[a]] < node_rank[nodes[b]]; });
      }
    }
    if (items.size() == 1) items.push_back(m);
    R.sd_depth.push_back(depth);
    for (size_t k = 1; k < items.size(); ++k) R.item_row.push_back(items[k]);
    R.sd_item.push_back((int64_t)R.item_row.size());
    std::vector<int32_t> perm(m);  // old local -> new local
    for (int64_t q = 0; q < m; ++q) perm[order[q]] = (int32_t)q;
    std::vector<int32_t> gn(m);
    for (int64_t q = 0; q < m; ++q) gn[perm[q]] = nodes[q];
    for (int64_t q = 0; q < m; ++q) loc[gn[q]] = (int32_t)q;

    // 4. local pattern of J_i^delta = R_i^delta J (R_i^delta)^T with its
    //    extraction map, extended by the symbolic level-of-fill ILU(k) pattern
    //    (fill blocks start at zero: gblk = -1)
    const int64_t r0 = R.sd_row.back();
    std::vector<std::vector<int32_t>> rcol(m);
    std::vector<std::vector<int32_t>> rlev(m);
    std::vector<std::vector<int64_t>> rgb(m);
    const int32_t END = (int32_t)m;  // list terminator, larger than every column
    std::vector<std::pair<int32_t, int64_t>> orig;
    for (int64_t q = 0; q < m; ++q) {
      int32_t v = gn[q];
      R.gnode.push_back(v);
      R.owned.push_back(owner[v] == s ? 1 : 0);
      // the row of J_i^delta (level 0), sorted by local column
      orig.clear();
      for (int64_t e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) {
        int32_t w = loc[P.col[e]];
        if (w >= 0) orig.push_back({w, e});
      }
      std::sort(orig.begin(), orig.end());
      int32_t head = END;
      for (size_t k = orig.size(); k-- > 0;) {
        const int32_t w = orig[k].first;
        nxt[w] = head;
        lev[w] = 0;
        src[w] = orig[k].second;
        head = w;
      }
      // level-of-fill: walk the L part in increasing column order (entries
      // created on the way are visited too) and merge each row k's U part,
      // level(q,j) = min over k of level(q,k) + level(k,j) + 1, kept if <= k_fill
      if (fill_level > 0) {
        for (int32_t k = head; k != END && k < q; k = nxt[k]) {
          const int32_t lqk = lev[k];
          int32_t prev = k;
          for (size_t f = 0; f < rcol[k].size(); ++f) {
            const int32_t j = rcol[k][f];
            if (j <= k) continue;
            const int32_t nl = lqk + rlev[k][f] + 1;
            if (nl > fill_level) continue;
            while (nxt[prev] < j) prev = nxt[prev];
            if (nxt[prev] == j) {
              if (nl < lev[j]) lev[j] = nl;
            } else {
              nxt[j] = nxt[prev];
              nxt[prev] = j;
              lev[j] = nl;
              src[j] = -1;
            }
            prev = j;
          }
        }
      }
      for (int32_t k = head; k != END; k = nxt[k]) {
        rcol[q].push_back(k);
        rlev[q].push_back(lev[k]);
        rgb[q].push_back(src[k]);
      }
    }
    for (int64_t q = 0; q < m; ++q) {
      for (size_t f = 0; f < rcol[q].size(); ++f) {
        if (rcol[q][f] == q) R.diag.push_back((int64_t)R.col.size());
        R.col.push_back((int32_t)(r0 + rcol[q][f]));
        R.gblk.push_back(rgb[q][f]);
      }
      R.row_ptr.push_back((int64_t)R.col.size());
    }
    // 5. ILU elimination lists and level schedules
    std::vector<int32_t> levL(m, 0), levU(m, 0);
    int32_t nlevL = 0, nlevU = 0;
    for (int64_t q = 0; q < m; ++q) {
      const int64_t rb = R.row_ptr[r0 + q], re = R.row_ptr[r0 + q + 1];
      for (int64_t e = rb; e < re; ++e) posq[R.col[e] - r0] = e;
      for (int64_t e = rb; e < re; ++e) {
        const int64_t k = R.col[e] - r0;
        if (k >= q) break;
        levL[q] = std::max(levL[q], levL[k] + 1);
        R.lent_pos.push_back(e);
        R.lent_kdiag.push_back(R.diag[r0 + k]);
        // updates A_qj -= A_qk A_kj for j > k in row k with (q, j) in the pattern,
        // in row k's column order
        const int64_t kb = R.row_ptr[r0 + k], ke = R.row_ptr[r0 + k + 1];
        for (int64_t f = kb; f < ke; ++f) {
          const int64_t j = R.col[f] - r0;
          if (j <= k) continue;
          const int64_t pq = posq[j];
          if (pq >= 0) {
            R.upd_tgt.push_back(pq);
            R.upd_src.push_back(f);
          }
        }
        R.upd_ptr.push_back((int64_t)R.upd_tgt.size());
      }
      for (int64_t e = rb; e < re; ++e) posq[R.col[e] - r0] = -1;
      R.lent_ptr.push_back((int64_t)R.lent_pos.size());
      nlevL = std::max(nlevL, levL[q] + 1);
    }
    for (int64_t q = m - 1; q >= 0; --q) {
      const int64_t rb = R.row_ptr[r0 + q], re = R.row_ptr[r0 + q + 1];
      for (int64_t e = rb; e < re; ++e) {
        const int64_t j = R.col[e] - r0;
        if (j > q) levU[q] = std::max(levU[q], levU[j] + 1);
      }
      nlevU = std::max(nlevU, levU[q] + 1);
    }
    auto emit_levels = [&](const std::vector<int32_t>& lev, int32_t nlev, std::vector<int64_t>& lptr,
                           std::vector<int32_t>& lrows, std::vector<int64_t>& sdl) {
      std::vector<int64_t> cnt(nlev + 1, 0);
      for (int64_t q = 0; q < m; ++q) cnt[lev[q] + 1]++;
      for (int32_t l = 0; l < nlev; ++l) cnt[l + 1] += cnt[l];
      const int64_t base = (int64_t)lrows.size();
      lrows.resize(base + m);
      std::vector<int64_t> f(cnt.begin(), cnt.end() - 1);
      for (int64_t q = 0; q < m; ++q) lrows[base + f[lev[q]]++] = (int32_t)q;
      for (int32_t l = 0; l < nlev; ++l) lptr.push_back(base + cnt[l + 1]);
      sdl.push_back((int64_t)lptr.size() - 1);
    };
    emit_levels(levL, nlevL, R.lvlL_ptr, R.lvlL_rows, R.sd_lvlL);
    emit_levels(levU, nlevU, R.lvlU_ptr, R.lvlU_rows, R.sd_lvlU);
    R.max_levels = std::max(R.max_levels, std::max(nlevL, nlevU));
    R.max_rows = std::max<int64_t>(R.max_rows, m);
    R.sd_row.push_back(r0 + m);
    for (int64_t q = 0; q < m; ++q) loc[gn[q]] = -1;
  }
  }  // omp parallel

  // concatenate: rows, blocks, L entries, updates and levels get the offsets of
  // the subdomains before them (sizes and offsets first, then the copies in
  // parallel, one subdomain per task)
  std::vector<int64_t> oR(np + 1, 0), oB(np + 1, 0), oL(np + 1, 0), oU(np + 1, 0);
  std::vector<int64_t> oLR(np + 1, 0), oUR(np + 1, 0), oLP(np + 1, 0), oUP(np + 1, 0), oI(np + 1, 0);
  for (int32_t s = 0; s < np; ++s) {
    const RasPlan& L = subs[s];
    oI[s + 1] = oI[s] + (int64_t)L.item_row.size();
    R.max_depth = std::max(R.max_depth, L.sd_depth.empty() ? 0 : L.sd_depth[0]);
    oR[s + 1] = oR[s] + (int64_t)L.gnode.size();
    oB[s + 1] = oB[s] + (int64_t)L.col.size();
    oL[s + 1] = oL[s] + (int64_t)L.lent_pos.size();
    oU[s + 1] = oU[s] + (int64_t)L.upd_tgt.size();
    oLR[s + 1] = oLR[s] + (int64_t)L.lvlL_rows.size();
    oUR[s + 1] = oUR[s] + (int64_t)L.lvlU_rows.size();
    oLP[s + 1] = oLP[s] + (int64_t)L.lvlL_ptr.size() - 1;
    oUP[s + 1] = oUP[s] + (int64_t)L.lvlU_ptr.size() - 1;
    R.max_levels = std::max(R.max_levels, L.max_levels);
    R.max_rows = std::max(R.max_rows, L.max_rows);
  }
  R.gnode.resize(oR[np]);
  R.owned.resize(oR[np]);
  R.diag.resize(oR[np]);
  R.row_ptr.assign(oR[np] + 1, 0);
  R.lent_ptr.assign(oR[np] + 1, 0);
  R.col.resize(oB[np]);
  R.gblk.resize(oB[np]);
  R.lent_pos.resize(oL[np]);
  R.lent_kdiag.resize(oL[np]);
  R.upd_ptr.assign(oL[np] + 1, 0);
  R.upd_tgt.resize(oU[np]);
  R.upd_src.resize(oU[np]);
  R.lvlL_rows.resize(oLR[np]);
  R.lvlU_rows.resize(oUR[np]);
  R.lvlL_ptr.assign(oLP[np] + 1, 0);
  R.lvlU_ptr.assign(oUP[np] + 1, 0);
  R.sd_row.assign(oR.begin(), oR.end());
  R.sd_item.assign(oI.begin(), oI.end());
  R.item_row.resize(oI[np]);
  R.sd_depth.resize(np);
  R.sd_lvlL.assign(oLP.begin(), oLP.end());
  R.sd_lvlU.assign(oUP.begin(), oUP.end());
#pragma omp parallel for schedule(dynamic, 4)
  for (int32_t s = 0; s < np; ++s) {
    RasPlan& L = subs[s];
    const int64_t RO = oR[s], BO = oB[s], LO = oL[s], UO = oU[s];
    const int64_t rows = oR[s + 1] - RO;
    for (int64_t i = 0; i < rows; ++i) {
      R.gnode[RO + i] = L.gnode[i];
      R.owned[RO + i] = L.owned[i];
      R.diag[RO + i] = L.diag[i] + BO;
      R.row_ptr[RO + i + 1] = L.row_ptr[i + 1] + BO;
      R.lent_ptr[RO + i + 1] = L.lent_ptr[i + 1] + LO;
    }
    for (size_t k = 0; k < L.col.size(); ++k) {
      R.col[BO + k] = (int32_t)(L.col[k] + RO);
      R.gblk[BO + k] = L.gblk[k];
    }
    for (size_t e = 0; e < L.lent_pos.size(); ++e) {
      R.lent_pos[LO + e] = L.lent_pos[e] + BO;
      R.lent_kdiag[LO + e] = L.lent_kdiag[e] + BO;
      R.upd_ptr[LO + e + 1] = L.upd_ptr[e + 1] + UO;
    }
    for (size_t u = 0; u < L.upd_tgt.size(); ++u) {
      R.upd_tgt[UO + u] = L.upd_tgt[u] + BO;
      R.upd_src[UO + u] = L.upd_src[u] + BO;
    }
    std::copy(L.item_row.begin(), L.item_row.end(), R.item_row.begin() + oI[s]);
    R.sd_depth[s] = L.sd_depth[0];
    std::copy(L.lvlL_rows.begin(), L.lvlL_rows.end(), R.lvlL_rows.begin() + oLR[s]);
    std::copy(L.lvlU_rows.begin(), L.lvlU_rows.end(), R.lvlU_rows.begin() + oUR[s]);
    for (size_t i = 1; i < L.lvlL_ptr.size(); ++i) R.lvlL_ptr[oLP[s] + i] = L.lvlL_ptr[i] + oLR[s];
    for (size_t i = 1; i < L.lvlU_ptr.size(); ++i) R.lvlU_ptr[oUP[s] + i] = L.lvlU_ptr[i] + oUR[s];
    L = RasPlan();  // release the per-subdomain memory early
  }
  R.np = np;
  return R;
}

}  // namespace fsi
