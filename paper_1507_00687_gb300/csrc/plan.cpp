// Host plan compiler: rule validation (Brent equations), principal
// quantities (Sec. 4.1), flattening of L levels into R^L leaf descriptors
// (Eq. 4.4), and the gradient rules obtained by the cyclic symmetry of the
// matrix-multiplication tensor (Sec. 5.3, App. A-C).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

#include <cuda_runtime.h>

#include "plan.h"

namespace fmm {

static int lin(int p, int q, int rows, int cols, int order) {
  return order == FMM_ORDER_ROW ? p * cols + q : q * rows + p;
}

fmm_status canonicalize(const fmm_rule& in, CanonRule* out) {
  if (in.m0 < 1 || in.k0 < 1 || in.n0 < 1 || in.r < 1) return FMM_ERR_ARG;
  if (in.m0 > 64 || in.k0 > 64 || in.n0 > 64 || in.r > 4096) return FMM_ERR_UNSUPPORTED;
  if (!in.U || !in.V || !in.W) return FMM_ERR_ARG;
  for (int o : {in.order_a, in.order_b, in.order_c})
    if (o != FMM_ORDER_ROW && o != FMM_ORDER_COL) return FMM_ERR_ARG;
  CanonRule c;
  c.m0 = in.m0; c.k0 = in.k0; c.n0 = in.n0; c.r = in.r;
  const int R = in.r;
  c.U.assign((size_t)in.m0 * in.k0 * R, 0.0);
  c.V.assign((size_t)in.k0 * in.n0 * R, 0.0);
  c.W.assign((size_t)in.m0 * in.n0 * R, 0.0);
  for (int p = 0; p < in.m0; ++p)
    for (int q = 0; q < in.k0; ++q)
      for (int r = 0; r < R; ++r)
        c.U[(size_t)(p * in.k0 + q) * R + r] = in.U[(size_t)lin(p, q, in.m0, in.k0, in.order_a) * R + r];
  for (int p = 0; p < in.k0; ++p)
    for (int q = 0; q < in.n0; ++q)
      for (int r = 0; r < R; ++r)
        c.V[(size_t)(p * in.n0 + q) * R + r] = in.V[(size_t)lin(p, q, in.k0, in.n0, in.order_b) * R + r];
  for (int p = 0; p < in.m0; ++p)
    for (int q = 0; q < in.n0; ++q)
      for (int r = 0; r < R; ++r)
        c.W[(size_t)(p * in.n0 + q) * R + r] = in.W[(size_t)lin(p, q, in.m0, in.n0, in.order_c) * R + r];
  for (double x : c.U) if (!std::isfinite(x)) return FMM_ERR_ARG;
  for (double x : c.V) if (!std::isfinite(x)) return FMM_ERR_ARG;
  for (double x : c.W) if (!std::isfinite(x)) return FMM_ERR_ARG;
  *out = std::move(c);
  return FMM_OK;
}

// The rule computes C = AB iff for all A entries (i,k), B entries (k2,j)
// and C entries (i2,j2):  sum_r U[(i,k),r] V[(k2,j),r] W[(i2,j2),r] equals
// 1 when i = i2, k = k2, j = j2 and 0 otherwise.  Coefficients are small
// dyadic rationals in practice, so the double sums are exact; a relative
// slack of 1e-9 admits other rationals.
int brent_violations(const CanonRule& c) {
  const int R = c.r;
  int bad = 0;
  for (int i = 0; i < c.m0; ++i)
    for (int k = 0; k < c.k0; ++k)
      for (int k2 = 0; k2 < c.k0; ++k2)
        for (int j = 0; j < c.n0; ++j)
          for (int i2 = 0; i2 < c.m0; ++i2)
            for (int j2 = 0; j2 < c.n0; ++j2) {
              double s = 0, mag = 0;
              for (int r = 0; r < R; ++r) {
                double t = c.U[(size_t)(i * c.k0 + k) * R + r] * c.V[(size_t)(k2 * c.n0 + j) * R + r] *
                           c.W[(size_t)(i2 * c.n0 + j2) * R + r];
                s += t;
                mag += std::fabs(t);
              }
              double want = (i == i2 && k == k2 && j == j2) ? 1.0 : 0.0;
              if (std::fabs(s - want) > 1e-9 * (1.0 + mag)) ++bad;
            }
  return bad;
}

// alpha_r, beta_r: nonzeros of column r of U, V; gamma_k: nonzeros of row k
// of W; a_r, b_r: column 1-norms (Eqs. 4.1-4.2).
// q_k = gamma_k + max_r (alpha_r + beta_r) [W_kr != 0], Q = max_k q_k (Def. 4.1).
// e_k = sum_r a_r b_r |W_kr|, E = max_k e_k (Def. 4.2).
void principal_quantities(CanonRule* c) {
  const int R = c->r, nA = c->m0 * c->k0, nB = c->k0 * c->n0, nC = c->m0 * c->n0;
  std::vector<double> alpha(R, 0), beta(R, 0), a(R, 0), b(R, 0);
  int64_t nnz = 0;
  for (int r = 0; r < R; ++r) {
    for (int i = 0; i < nA; ++i) {
      double u = c->U[(size_t)i * R + r];
      if (u != 0) { alpha[r] += 1; ++nnz; }
      a[r] += std::fabs(u);
    }
    for (int j = 0; j < nB; ++j) {
      double v = c->V[(size_t)j * R + r];
      if (v != 0) { beta[r] += 1; ++nnz; }
      b[r] += std::fabs(v);
    }
  }
  double Q = 0, E = 0;
  c->gamma.assign(nC, 0.0);
  for (int k = 0; k < nC; ++k) {
    double gamma = 0, mx = 0, e = 0;
    for (int r = 0; r < R; ++r) {
      double w = c->W[(size_t)k * R + r];
      if (w != 0) {
        gamma += 1;
        ++nnz;
        mx = std::max(mx, alpha[r] + beta[r]);
      }
      e += a[r] * b[r] * std::fabs(w);
    }
    Q = std::max(Q, gamma + mx);
    E = std::max(E, e);
    c->gamma[k] = gamma;
  }
  c->alpha = alpha;
  c->beta = beta;
  c->a = a;
  c->b = b;
  c->Q = Q;
  c->E = E;
  c->nnz = nnz;
}

namespace {

struct Term {
  int32_t row, col;
  double coef;
};

// All (i_1..i_L) with prod_l X_l[i_l, r_l] != 0, in lexicographic order of
// (i_1, ..., i_L) (level 1 slowest), with the block position
// row = sum_l p_l prod_{l' > l} rows_{l'}, col likewise.
void expand(const std::vector<const std::vector<double>*>& X, const std::vector<int>& rows,
            const std::vector<int>& cols, const std::vector<int>& R, const std::vector<int>& rl,
            int level, int32_t row, int32_t col, double coef, std::vector<Term>* out) {
  const int L = (int)X.size();
  if (level == L) {
    out->push_back({row, col, coef});
    return;
  }
  const int nr = rows[level], nc = cols[level];
  for (int i = 0; i < nr * nc; ++i) {
    double x = (*X[level])[(size_t)i * R[level] + rl[level]];
    if (x == 0) continue;
    expand(X, rows, cols, R, rl, level + 1, row * nr + i / nc, col * nc + i % nc, coef * x, out);
  }
}


// Append one leaf's flattened terms to p->host; leaves arrive in order.
// touched: the C blocks some earlier leaf adds into.
void add_leaf(Plan* p, int64_t leaf, const std::vector<Term>& ta, const std::vector<Term>& tb,
              const std::vector<Term>& tc, std::set<int32_t>* touched) {
  p->max_terms = std::max(p->max_terms, (int)std::max(ta.size(), std::max(tb.size(), tc.size())));
  p->nnz += (int64_t)(ta.size() + tb.size() + tc.size());
  LeafDesc& d = p->host[(size_t)leaf];
  std::memset(&d, 0, sizeof(d));
  if ((int)ta.size() > kMaxTerms || (int)tb.size() > kMaxTerms || (int)tc.size() > kMaxTerms) return;
  d.na = (int)ta.size();
  d.nb = (int)tb.size();
  d.nc = (int)tc.size();
  for (int t = 0; t < d.na; ++t) { d.a_blk[t] = (ta[t].row << 16) | ta[t].col; d.a_coef[t] = (float)ta[t].coef; }
  for (int t = 0; t < d.nb; ++t) { d.b_blk[t] = (tb[t].row << 16) | tb[t].col; d.b_coef[t] = (float)tb[t].coef; }
  for (int t = 0; t < d.nc; ++t) {
    int32_t blk = (tc[t].row << 16) | tc[t].col;
    d.c_blk[t] = blk;
    d.c_coef[t] = (float)tc[t].coef;
    d.c_first[t] = touched->insert(blk).second ? 1 : 0;
  }
}

// The compact per-side term lists from p->host.
void build_lists(Plan* p) {
  for (int side = 0; side < 3; ++side) {
    int64_t nnz = 0;
    for (const LeafDesc& d : p->host) nnz += side == 0 ? d.na : side == 1 ? d.nb : d.nc;
    p->list_off[side] = (int64_t)p->lists.size();
    p->list_nnz[side] = nnz;
    const size_t base = p->lists.size();
    p->lists.resize(base + (size_t)(p->leaves + 1 + 2 * nnz));
    int32_t* start = p->lists.data() + base;
    int32_t* blk = start + p->leaves + 1;
    int32_t* coef = blk + nnz;
    int64_t at = 0;
    for (int64_t r = 0; r < p->leaves; ++r) {
      const LeafDesc& d = p->host[(size_t)r];
      start[r] = (int32_t)at;
      const int n = side == 0 ? d.na : side == 1 ? d.nb : d.nc;
      for (int t = 0; t < n; ++t, ++at) {
        const float c = side == 0 ? d.a_coef[t] : side == 1 ? d.b_coef[t] : d.c_coef[t];
        blk[at] = side == 0 ? d.a_blk[t] : side == 1 ? d.b_blk[t] : (d.c_blk[t] | (d.c_first[t] ? kFirstBit : 0));
        std::memcpy(&coef[at], &c, 4);
      }
    }
    start[p->leaves] = (int32_t)at;
  }
  // per-C-block lists, leaves in order
  const int64_t nblk = p->pm * p->pn;
  if (nblk > kMaxGatherBlocks) return;
  std::vector<int32_t> count((size_t)nblk + 1, 0);
  for (const LeafDesc& d : p->host)
    for (int t = 0; t < d.nc; ++t) ++count[(size_t)((d.c_blk[t] >> 16) * p->pn + (d.c_blk[t] & 0xFFFF)) + 1];
  for (int64_t k = 0; k < nblk; ++k) count[(size_t)k + 1] += count[(size_t)k];
  const int64_t nnz = p->list_nnz[2];
  p->gather_off = (int64_t)p->lists.size();
  p->lists.resize(p->lists.size() + (size_t)(nblk + 1 + 2 * nnz));
  int32_t* gstart = p->lists.data() + p->gather_off;
  int32_t* gleaf = gstart + nblk + 1;
  int32_t* gcoef = gleaf + nnz;
  std::copy(count.begin(), count.end(), gstart);
  for (int64_t r = 0; r < p->leaves; ++r) {
    const LeafDesc& d = p->host[(size_t)r];
    for (int t = 0; t < d.nc; ++t) {
      const int64_t k = (d.c_blk[t] >> 16) * p->pn + (d.c_blk[t] & 0xFFFF);
      const int32_t at = count[(size_t)k]++;
      gleaf[at] = (int32_t)r;
      std::memcpy(&gcoef[at], &d.c_coef[t], 4);
    }
  }
}

bool valid_leaf_format(int leaf_format) {
  return leaf_format == FMM_LEAF_BF16 || leaf_format == FMM_LEAF_F16 || leaf_format == FMM_LEAF_BF16X3 ||
         leaf_format == FMM_LEAF_E4M3B128;
}

// The leaves of one root-to-leaf path: X[l] is the path's U (V, W) at
// level l+1, R[l] that rule's rank, rl[l] the product index taken there.
struct Path {
  std::vector<const std::vector<double>*> U, V, W;
  std::vector<int> m0, k0, n0, R, rl;
};

void expand_path(const Path& q, std::vector<Term>* ta, std::vector<Term>* tb, std::vector<Term>* tc) {
  ta->clear(); tb->clear(); tc->clear();
  expand(q.U, q.m0, q.k0, q.R, q.rl, 0, 0, 0, 1.0, ta);
  expand(q.V, q.k0, q.n0, q.R, q.rl, 0, 0, 0, 1.0, tb);
  expand(q.W, q.m0, q.n0, q.R, q.rl, 0, 0, 0, 1.0, tc);
}

// Node layout of a tree plan: level_start[l] is the index in node_rule of
// level l's first node, first_child[i] the index of node i's first child.
struct TreeIndex {
  std::vector<int64_t> level_start, first_child;
};

// max_k delta_k over the C blocks below `node` (Sec. 4.5): at a node,
// delta_k = gamma_{k_l} + max over r with W[k_l, r] != 0 of the child's
// delta, with chi (the sum of alpha_r + beta_r along the path) at the leaves.
// The max over k splits into the max over k_l of gamma plus the children's
// maxima.
double tree_delta_max(const Plan& p, const TreeIndex& t, int64_t node, int level, double chi) {
  if (level == p.levels) return chi;
  const CanonRule& c = p.table[(size_t)p.node_rule[(size_t)node]];
  std::vector<double> sub((size_t)c.r);
  for (int r = 0; r < c.r; ++r)
    sub[(size_t)r] = tree_delta_max(p, t, t.first_child[(size_t)node] + r, level + 1, chi + c.alpha[r] + c.beta[r]);
  double best = 0;
  for (int k = 0; k < c.m0 * c.n0; ++k) {
    double mx = -1;
    for (int r = 0; r < c.r; ++r)
      if (c.W[(size_t)k * c.r + r] != 0) mx = std::max(mx, sub[(size_t)r]);
    if (mx >= 0) best = std::max(best, c.gamma[k] + mx);
  }
  return best;
}

// xi_k over the flattened C blocks below `node` (k_l slowest, Sec. 4.5):
// xi_k = sum_r |W[k_l, r]| a_r b_r xi^{child r}_{k_{l+1}..}, 1 at the leaves.
std::vector<double> tree_xi(const Plan& p, const TreeIndex& t, int64_t node, int level) {
  if (level == p.levels) return {1.0};
  const CanonRule& c = p.table[(size_t)p.node_rule[(size_t)node]];
  std::vector<std::vector<double>> sub((size_t)c.r);
  for (int r = 0; r < c.r; ++r) sub[(size_t)r] = tree_xi(p, t, t.first_child[(size_t)node] + r, level + 1);
  const size_t n = sub[0].size();
  std::vector<double> out((size_t)(c.m0 * c.n0) * n, 0.0);
  for (int k = 0; k < c.m0 * c.n0; ++k)
    for (int r = 0; r < c.r; ++r) {
      const double w = std::fabs(c.W[(size_t)k * c.r + r]);
      if (w == 0) continue;
      for (size_t j = 0; j < n; ++j) out[(size_t)k * n + j] += w * c.a[r] * c.b[r] * sub[(size_t)r][j];
    }
  return out;
}

// Depth-first walk over the tree's leaves (product r = 0..R-1 at every
// node, so leaves come in the order the uniform enumeration uses).
void tree_leaves(Plan* p, const TreeIndex& t, int64_t node, int level, Path* q, int64_t* leaf,
                 std::vector<Term>* ta, std::vector<Term>* tb, std::vector<Term>* tc, std::set<int32_t>* touched) {
  if (level == p->levels) {
    expand_path(*q, ta, tb, tc);
    add_leaf(p, (*leaf)++, *ta, *tb, *tc, touched);
    return;
  }
  const CanonRule& c = p->table[(size_t)p->node_rule[(size_t)node]];
  q->U[(size_t)level] = &c.U;
  q->V[(size_t)level] = &c.V;
  q->W[(size_t)level] = &c.W;
  q->R[(size_t)level] = c.r;
  for (int r = 0; r < c.r; ++r) {
    q->rl[(size_t)level] = r;
    tree_leaves(p, t, t.first_child[(size_t)node] + r, level + 1, q, leaf, ta, tb, tc, touched);
  }
}

}  // namespace

fmm_status build_plan(const std::vector<CanonRule>& rules_in, int leaf_format, Plan** out) {
  if (!valid_leaf_format(leaf_format)) return FMM_ERR_ARG;
  Plan* p = new Plan();
  p->levels = (int)rules_in.size();
  p->leaf_format = leaf_format;
  p->rules = rules_in;
  for (auto& r : p->rules) {
    if (brent_violations(r) != 0) {
      delete p;
      return FMM_ERR_NOT_MATMUL;
    }
    principal_quantities(&r);
    p->pm *= r.m0;
    p->pk *= r.k0;
    p->pn *= r.n0;
    p->leaves *= r.r;
    p->q_sum += r.Q;
    p->e_prod *= r.E;
    if (p->pm > 32768 || p->pk > 32768 || p->pn > 32768 || p->leaves > 1000000) {
      delete p;
      return FMM_ERR_UNSUPPORTED;
    }
  }
  const int L = p->levels;
  Path q;
  for (auto& r : p->rules) {
    q.U.push_back(&r.U); q.V.push_back(&r.V); q.W.push_back(&r.W);
    q.m0.push_back(r.m0); q.k0.push_back(r.k0); q.n0.push_back(r.n0); q.R.push_back(r.r);
  }
  q.rl.assign(L, 0);
  p->host.resize((size_t)p->leaves);
  std::set<int32_t> touched;
  std::vector<Term> ta, tb, tc;
  for (int64_t leaf = 0; leaf < p->leaves; ++leaf) {
    // leaf = sum_l r_l prod_{l' > l} R_{l'}  (level 1 slowest)
    int64_t rem = leaf;
    for (int l = L - 1; l >= 0; --l) {
      q.rl[l] = (int)(rem % q.R[l]);
      rem /= q.R[l];
    }
    expand_path(q, &ta, &tb, &tc);
    add_leaf(p, leaf, ta, tb, tc, &touched);
  }
  build_lists(p);
  *out = p;
  return FMM_OK;
}

fmm_status build_tree_plan(const std::vector<CanonRule>& table_in, int levels, const std::vector<int>& node_rule,
                           int leaf_format, Plan** out) {
  if (!valid_leaf_format(leaf_format) || levels < 1 || table_in.empty()) return FMM_ERR_ARG;
  Plan* p = new Plan();
  p->levels = levels;
  p->leaf_format = leaf_format;
  p->table = table_in;
  p->node_rule = node_rule;
  for (auto& r : p->table) {
    if (brent_violations(r) != 0) {
      delete p;
      return FMM_ERR_NOT_MATMUL;
    }
    principal_quantities(&r);
  }
  // Level by level: the nodes of level l+1 are the children of level l's
  // nodes, R of them per node, in node order.
  TreeIndex t;
  t.first_child.assign(node_rule.size(), -1);
  int64_t at = 0, count = 1;
  for (int l = 0; l < levels; ++l) {
    t.level_start.push_back(at);
    if (at + count > (int64_t)node_rule.size()) {
      delete p;
      return FMM_ERR_ARG;
    }
    int64_t next = 0;
    const CanonRule* first = nullptr;
    for (int64_t i = at; i < at + count; ++i) {
      const int ri = node_rule[(size_t)i];
      if (ri < 0 || ri >= (int)p->table.size()) {
        delete p;
        return FMM_ERR_ARG;
      }
      const CanonRule& c = p->table[(size_t)ri];
      if (!first) first = &c;
      // every path partitions A, B and C alike
      if (c.m0 != first->m0 || c.k0 != first->k0 || c.n0 != first->n0) {
        delete p;
        return FMM_ERR_ARG;
      }
      if (c.r != first->r) p->level_r_uniform = false;
      t.first_child[(size_t)i] = at + count + next;
      next += c.r;
      if (next > 1000000) {
        delete p;
        return FMM_ERR_UNSUPPORTED;
      }
    }
    p->rules.push_back(*first);
    p->pm *= first->m0;
    p->pk *= first->k0;
    p->pn *= first->n0;
    at += count;
    count = next;
    if (p->pm > 32768 || p->pk > 32768 || p->pn > 32768) {
      delete p;
      return FMM_ERR_UNSUPPORTED;
    }
  }
  if (at != (int64_t)node_rule.size()) {
    delete p;
    return FMM_ERR_ARG;
  }
  p->leaves = count;
  p->q_sum = tree_delta_max(*p, t, 0, 0, 0.0);
  if (p->pm * p->pn <= (int64_t)1 << 22) {
    const std::vector<double> xi = tree_xi(*p, t, 0, 0);
    p->e_prod = *std::max_element(xi.begin(), xi.end());
  } else {
    // too many C blocks to list: the product over levels of the largest E
    // of the level's rules bounds every xi_k
    p->e_prod = 1;
    for (int l = 0; l < levels; ++l) {
      double e = 0;
      const int64_t end = l + 1 < levels ? t.level_start[(size_t)l + 1] : (int64_t)node_rule.size();
      for (int64_t i = t.level_start[(size_t)l]; i < end; ++i) e = std::max(e, p->table[(size_t)node_rule[(size_t)i]].E);
      p->e_prod *= e;
    }
  }
  Path q;
  q.U.assign(levels, nullptr); q.V.assign(levels, nullptr); q.W.assign(levels, nullptr);
  q.R.assign(levels, 0); q.rl.assign(levels, 0);
  for (auto& r : p->rules) { q.m0.push_back(r.m0); q.k0.push_back(r.k0); q.n0.push_back(r.n0); }
  p->host.resize((size_t)p->leaves);
  std::set<int32_t> touched;
  std::vector<Term> ta, tb, tc;
  int64_t leaf = 0;
  tree_leaves(p, t, 0, 0, &q, &leaf, &ta, &tb, &tc, &touched);
  build_lists(p);
  *out = p;
  return FMM_OK;
}

void destroy_plan(Plan* p) {
  if (!p) return;
  if (p->dev) cudaFree(p->dev);
  destroy_plan(p->level1);
  destroy_plan(p->grad_a);
  destroy_plan(p->grad_b);
  delete p;
}

// Row (p, q) of a row-major rows x cols operand -> row (q, p) of the
// row-major transpose.
static std::vector<double> transpose_rows(const std::vector<double>& X, int rows, int cols, int R) {
  std::vector<double> out(X.size());
  for (int p = 0; p < rows; ++p)
    for (int q = 0; q < cols; ++q)
      for (int r = 0; r < R; ++r) out[(size_t)(q * rows + p) * R + r] = X[(size_t)(p * cols + q) * R + r];
  return out;
}

// dA = dC B^T is an <m0, n0, k0> product: tr-form symmetry maps the dC
// operand to W, B^T to V with transposed indexing, and dA to U.
CanonRule rule_for_grad_a(const CanonRule& c) {
  CanonRule g;
  g.m0 = c.m0; g.k0 = c.n0; g.n0 = c.k0; g.r = c.r;
  g.U = c.W;
  g.V = transpose_rows(c.V, c.k0, c.n0, c.r);
  g.W = c.U;
  return g;
}

// dB = A^T dC is a <k0, m0, n0> product: A^T takes U with transposed
// indexing, dC takes W, and dB takes V.
CanonRule rule_for_grad_b(const CanonRule& c) {
  CanonRule g;
  g.m0 = c.k0; g.k0 = c.m0; g.n0 = c.n0; g.r = c.r;
  g.U = transpose_rows(c.U, c.m0, c.k0, c.r);
  g.V = c.W;
  g.W = c.V;
  return g;
}

}  // namespace fmm
