// Host plan compiler: rule validation (Brent equations), principal
// quantities (Sec. 4.1), flattening of L levels into R^L leaf descriptors
// (Eq. 4.4), and the gradient rules obtained by the cyclic symmetry of the
// matrix-multiplication tensor (Sec. 5.3, App. A-C).
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
  }
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

}  // namespace

fmm_status build_plan(const std::vector<CanonRule>& rules_in, int leaf_format, Plan** out) {
  if (leaf_format != FMM_LEAF_BF16 && leaf_format != FMM_LEAF_F16 && leaf_format != FMM_LEAF_BF16X3 &&
      leaf_format != FMM_LEAF_E4M3B128)
    return FMM_ERR_ARG;
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
  std::vector<const std::vector<double>*> Us, Vs, Ws;
  std::vector<int> m0s, k0s, n0s, Rs;
  for (auto& r : p->rules) {
    Us.push_back(&r.U); Vs.push_back(&r.V); Ws.push_back(&r.W);
    m0s.push_back(r.m0); k0s.push_back(r.k0); n0s.push_back(r.n0); Rs.push_back(r.r);
  }
  p->host.resize((size_t)p->leaves);
  std::set<int32_t> touched;
  std::vector<int> rl(L, 0);
  std::vector<Term> ta, tb, tc;
  for (int64_t leaf = 0; leaf < p->leaves; ++leaf) {
    // leaf = sum_l r_l prod_{l' > l} R_{l'}  (level 1 slowest)
    int64_t rem = leaf;
    for (int l = L - 1; l >= 0; --l) {
      rl[l] = (int)(rem % Rs[l]);
      rem /= Rs[l];
    }
    ta.clear(); tb.clear(); tc.clear();
    expand(Us, m0s, k0s, Rs, rl, 0, 0, 0, 1.0, &ta);
    expand(Vs, k0s, n0s, Rs, rl, 0, 0, 0, 1.0, &tb);
    expand(Ws, m0s, n0s, Rs, rl, 0, 0, 0, 1.0, &tc);
    p->max_terms = std::max(p->max_terms, (int)std::max(ta.size(), std::max(tb.size(), tc.size())));
    p->nnz += (int64_t)(ta.size() + tb.size() + tc.size());
    LeafDesc& d = p->host[(size_t)leaf];
    std::memset(&d, 0, sizeof(d));
    if ((int)ta.size() > kMaxTerms || (int)tb.size() > kMaxTerms || (int)tc.size() > kMaxTerms) continue;
    d.na = (int)ta.size();
    d.nb = (int)tb.size();
    d.nc = (int)tc.size();
    for (int t = 0; t < d.na; ++t) { d.a_blk[t] = (ta[t].row << 16) | ta[t].col; d.a_coef[t] = (float)ta[t].coef; }
    for (int t = 0; t < d.nb; ++t) { d.b_blk[t] = (tb[t].row << 16) | tb[t].col; d.b_coef[t] = (float)tb[t].coef; }
    for (int t = 0; t < d.nc; ++t) {
      int32_t blk = (tc[t].row << 16) | tc[t].col;
      d.c_blk[t] = blk;
      d.c_coef[t] = (float)tc[t].coef;
      d.c_first[t] = touched.insert(blk).second ? 1 : 0;
    }
  }
  // compact per-side term lists
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
