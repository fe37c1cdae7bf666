// Rule algebra (host): new base-case rules from old ones, every result
// checked against the Brent equations.
//
//  - rotation: the cyclic symmetry of the matrix-multiplication tensor
//    (App. A-B): [[W, U, V]] of a <m0,k0,n0> rule is a <n0,m0,k0> rule;
//  - composition: two recursion steps as one rule (Eq. 4.4 with L = 2);
//  - transformation [[XU U, XV V, XW W]] (Sec. 3.4, the form of the D'Alberto
//    and Castrapel-Gustafson variants);
//  - permutation of the block indices i, k, j (the Kronecker factors of the
//    variants of Sec. 3.4 are such permutations);
//  - the recursion trees of the Castrapel-Gustafson variants (Sec. 3.4):
//    random, round-robin and matrix-dependent selection per node.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.h"
#include "rules.h"

namespace fmm {

// Write a canonical (row-major A, B, C) rule into caller arrays.
static void emit(const CanonRule& c, double* U, double* V, double* W, fmm_rule* out) {
  std::memcpy(U, c.U.data(), c.U.size() * sizeof(double));
  std::memcpy(V, c.V.data(), c.V.size() * sizeof(double));
  std::memcpy(W, c.W.data(), c.W.size() * sizeof(double));
  out->m0 = c.m0;
  out->k0 = c.k0;
  out->n0 = c.n0;
  out->r = c.r;
  out->U = U;
  out->V = V;
  out->W = W;
  out->order_a = out->order_b = out->order_c = FMM_ORDER_ROW;
}

static fmm_status valid(const fmm_rule& in, CanonRule* c) {
  fmm_status s = canonicalize(in, c);
  if (s != FMM_OK) return s;
  return brent_violations(*c) ? FMM_ERR_NOT_MATMUL : FMM_OK;
}

fmm_status rule_rotate(const fmm_rule& in, double* U, double* V, double* W, fmm_rule* out) {
  CanonRule c;
  fmm_status s = valid(in, &c);
  if (s != FMM_OK) return s;
  // sum_(i,k,j) a_ik b_kj c_ij read with the factors cycled: a new A entry
  // (j, i) is C's (i, j), a new B entry (i, k) is A's, a new C entry (j, k)
  // is B's (k, j).
  const int m = c.m0, k = c.k0, n = c.n0, R = c.r;
  CanonRule o;
  o.m0 = n;
  o.k0 = m;
  o.n0 = k;
  o.r = R;
  o.U.assign((size_t)n * m * R, 0.0);
  o.V.assign((size_t)m * k * R, 0.0);
  o.W.assign((size_t)n * k * R, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j)
      for (int r = 0; r < R; ++r) o.U[(size_t)(j * m + i) * R + r] = c.W[(size_t)(i * n + j) * R + r];
  o.V = c.U;
  for (int kk = 0; kk < k; ++kk)
    for (int j = 0; j < n; ++j)
      for (int r = 0; r < R; ++r) o.W[(size_t)(j * k + kk) * R + r] = c.V[(size_t)(kk * n + j) * R + r];
  if (brent_violations(o)) return FMM_ERR_NOT_MATMUL;
  emit(o, U, V, W, out);
  return FMM_OK;
}

fmm_status rule_compose(const fmm_rule& outer, const fmm_rule& inner, double* U, double* V, double* W,
                        fmm_rule* out) {
  CanonRule a, b;
  fmm_status s = valid(outer, &a);
  if (s != FMM_OK) return s;
  if ((s = valid(inner, &b)) != FMM_OK) return s;
  if ((int64_t)a.m0 * b.m0 > 64 || (int64_t)a.k0 * b.k0 > 64 || (int64_t)a.n0 * b.n0 > 64 ||
      (int64_t)a.r * b.r > 4096)
    return FMM_ERR_UNSUPPORTED;
  CanonRule o;
  o.m0 = a.m0 * b.m0;
  o.k0 = a.k0 * b.k0;
  o.n0 = a.n0 * b.n0;
  o.r = a.r * b.r;
  // Entry (p1, q1) of the outer split then (p2, q2) of the inner one is
  // entry (p1 rows2 + p2, q1 cols2 + q2) of the composite operand, and
  // product (r1, r2) = r1 R2 + r2 has coefficient X1[(p1,q1),r1] X2[(p2,q2),r2].
  auto flat = [&](const std::vector<double>& X1, int rows1, int cols1, int R1, const std::vector<double>& X2,
                  int rows2, int cols2, int R2, std::vector<double>* Y) {
    const int cols = cols1 * cols2;
    Y->assign((size_t)rows1 * rows2 * cols * R1 * R2, 0.0);
    for (int p1 = 0; p1 < rows1; ++p1)
      for (int q1 = 0; q1 < cols1; ++q1)
        for (int p2 = 0; p2 < rows2; ++p2)
          for (int q2 = 0; q2 < cols2; ++q2) {
            const size_t row = (size_t)(p1 * rows2 + p2) * cols + q1 * cols2 + q2;
            for (int r1 = 0; r1 < R1; ++r1)
              for (int r2 = 0; r2 < R2; ++r2)
                (*Y)[row * R1 * R2 + (size_t)r1 * R2 + r2] =
                    X1[(size_t)(p1 * cols1 + q1) * R1 + r1] * X2[(size_t)(p2 * cols2 + q2) * R2 + r2];
          }
  };
  flat(a.U, a.m0, a.k0, a.r, b.U, b.m0, b.k0, b.r, &o.U);
  flat(a.V, a.k0, a.n0, a.r, b.V, b.k0, b.n0, b.r, &o.V);
  flat(a.W, a.m0, a.n0, a.r, b.W, b.m0, b.n0, b.r, &o.W);
  if (brent_violations(o)) return FMM_ERR_NOT_MATMUL;
  emit(o, U, V, W, out);
  return FMM_OK;
}

fmm_status rule_transform(const fmm_rule& in, const double* XU, const double* XV, const double* XW, double* U,
                          double* V, double* W, fmm_rule* out) {
  CanonRule c;
  fmm_status s = valid(in, &c);
  if (s != FMM_OK) return s;
  if (!XU || !XV || !XW) return FMM_ERR_ARG;
  // X (n x n) times the rule's own table (n x R), in the rule's entry order
  const int R = in.r;
  auto mix = [&](const double* X, const double* T, int nrow, std::vector<double>* Y) {
    Y->assign((size_t)nrow * R, 0.0);
    for (int i = 0; i < nrow; ++i)
      for (int t = 0; t < nrow; ++t) {
        const double x = X[(size_t)i * nrow + t];
        if (x == 0) continue;
        for (int r = 0; r < R; ++r) (*Y)[(size_t)i * R + r] += x * T[(size_t)t * R + r];
      }
  };
  std::vector<double> u, v, w;
  mix(XU, in.U, in.m0 * in.k0, &u);
  mix(XV, in.V, in.k0 * in.n0, &v);
  mix(XW, in.W, in.m0 * in.n0, &w);
  fmm_rule t = in;
  t.U = u.data();
  t.V = v.data();
  t.W = w.data();
  CanonRule o;
  if ((s = valid(t, &o)) != FMM_OK) return s;
  emit(o, U, V, W, out);
  return FMM_OK;
}

static bool is_perm(const int32_t* p, int n) {
  std::vector<char> seen(n, 0);
  for (int i = 0; i < n; ++i) {
    if (p[i] < 0 || p[i] >= n || seen[p[i]]) return false;
    seen[p[i]] = 1;
  }
  return true;
}

// U'[(i,k)] = U[(pi(i), pk(k))], V'[(k,j)] = V[(pk(k), pj(j))],
// W'[(i,j)] = W[(pi(i), pj(j))]: the rule applied to the blocks of A, B
// relabelled by the permutations, with C's blocks relabelled back, so it
// computes the same product.
static CanonRule permute_canon(const CanonRule& c, const int32_t* pi, const int32_t* pk, const int32_t* pj) {
  CanonRule o = c;
  const int R = c.r;
  for (int i = 0; i < c.m0; ++i)
    for (int k = 0; k < c.k0; ++k)
      for (int r = 0; r < R; ++r) o.U[(size_t)(i * c.k0 + k) * R + r] = c.U[(size_t)(pi[i] * c.k0 + pk[k]) * R + r];
  for (int k = 0; k < c.k0; ++k)
    for (int j = 0; j < c.n0; ++j)
      for (int r = 0; r < R; ++r) o.V[(size_t)(k * c.n0 + j) * R + r] = c.V[(size_t)(pk[k] * c.n0 + pj[j]) * R + r];
  for (int i = 0; i < c.m0; ++i)
    for (int j = 0; j < c.n0; ++j)
      for (int r = 0; r < R; ++r) o.W[(size_t)(i * c.n0 + j) * R + r] = c.W[(size_t)(pi[i] * c.n0 + pj[j]) * R + r];
  return o;
}

fmm_status rule_permute(const fmm_rule& in, const int32_t* pi, const int32_t* pk, const int32_t* pj, double* U,
                        double* V, double* W, fmm_rule* out) {
  CanonRule c;
  fmm_status s = valid(in, &c);
  if (s != FMM_OK) return s;
  if (!pi || !pk || !pj) return FMM_ERR_ARG;
  if (!is_perm(pi, c.m0) || !is_perm(pk, c.k0) || !is_perm(pj, c.n0)) return FMM_ERR_ARG;
  CanonRule o = permute_canon(c, pi, pk, pj);
  if (brent_violations(o)) return FMM_ERR_NOT_MATMUL;
  emit(o, U, V, W, out);
  return FMM_OK;
}

// Variant v = 0..7 of a <2,2,2> rule (Sec. 3.4, Castrapel-Gustafson):
// [[(P^x (x) P^y) U, (P^z (x) P^x) V, (P^y (x) P^z) W]] with P the 2 x 2
// exchange, in the paper's entry order (A, B column-major, C row-major).
// There the first Kronecker factor acts on the column index of A and B and
// on the row index of C, so P^x exchanges the k blocks, P^y the i blocks
// and P^z the j blocks.  x = 1 when bit 1 of v is set (else 2: P^2 = I),
// y = 1 when bit 0 is set, z = 1 when bit 2 is set; v = 0 is the rule.
CanonRule cg_variant(const CanonRule& c, int v) {
  const int32_t id[2] = {0, 1}, sw[2] = {1, 0};
  return permute_canon(c, (v & 1) ? sw : id, (v & 2) ? sw : id, (v & 4) ? sw : id);
}

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the output for counter value n of stream
// `seed` is the mix of seed + (n + 1) * golden gamma.
uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

namespace {

// Bounds on the max-abs of the finest blocks of one operand of a node: a
// g x g grid (g = 2^(levels below and at this node)), row-major.
struct Bounds {
  int g;
  std::vector<double> v;
  double at(int p, int q) const { return v[(size_t)p * g + q]; }
};

// Max over the finest blocks inside quadrant (p, q) of a node's operand.
double quadrant_max(const Bounds& b, int p, int q) {
  const int h = b.g / 2;
  double m = 0;
  for (int s = 0; s < h; ++s)
    for (int t = 0; t < h; ++t) m = std::max(m, b.at(p * h + s, q * h + t));
  return m;
}

// Growth estimate of one node under rule c: max over C blocks k of
// sum_r |W_kr| (sum_i |U_ir| alpha_i) (sum_j |V_jr| beta_j), with alpha_i,
// beta_j the quadrant bounds of the node's operands (the norm-wise growth
// of the proof of Theorem 4.1 for one level, on the actual blocks).  Sums
// in ascending index order.
double node_cost(const CanonRule& c, const Bounds& A, const Bounds& B) {
  const int R = c.r;
  double qa[4], qb[4];
  for (int i = 0; i < 4; ++i) {
    qa[i] = quadrant_max(A, i / 2, i % 2);
    qb[i] = quadrant_max(B, i / 2, i % 2);
  }
  std::vector<double> sa(R), sb(R);
  for (int r = 0; r < R; ++r) {
    double x = 0, y = 0;
    for (int i = 0; i < 4; ++i) x += std::fabs(c.U[(size_t)i * R + r]) * qa[i];
    for (int j = 0; j < 4; ++j) y += std::fabs(c.V[(size_t)j * R + r]) * qb[j];
    sa[r] = x;
    sb[r] = y;
  }
  double worst = 0;
  for (int k = 0; k < 4; ++k) {
    double e = 0;
    for (int r = 0; r < R; ++r) e += std::fabs(c.W[(size_t)k * R + r]) * (sa[r] * sb[r]);
    worst = std::max(worst, e);
  }
  return worst;
}

// Bounds of the operand S_r (T_r) of product r one level down: each finest
// block of S_r is sum_i U_ir times the same-position block of quadrant i,
// so its max-abs is at most sum_i |U_ir| times theirs.
Bounds child_bounds(const CanonRule& c, const Bounds& X, int r, bool a_side) {
  const int R = c.r, h = X.g / 2;
  Bounds o;
  o.g = h;
  o.v.assign((size_t)h * h, 0.0);
  const std::vector<double>& T = a_side ? c.U : c.V;
  for (int s = 0; s < h; ++s)
    for (int t = 0; t < h; ++t) {
      double acc = 0;
      for (int i = 0; i < 4; ++i) acc += std::fabs(T[(size_t)i * R + r]) * X.at((i / 2) * h + s, (i % 2) * h + t);
      o.v[(size_t)s * h + t] = acc;
    }
  return o;
}

}  // namespace

fmm_status cg_select(const CanonRule& base, int levels, int selection, uint64_t seed, const float* block_max_a,
                     const float* block_max_b, std::vector<int>* node_rule) {
  if (base.m0 != 2 || base.k0 != 2 || base.n0 != 2) return FMM_ERR_UNSUPPORTED;
  if (levels < 1 || levels > 8) return FMM_ERR_ARG;
  const int R = base.r;
  int64_t nodes = 0, width = 1;
  for (int l = 0; l < levels; ++l) {
    nodes += width;
    width *= R;
    if (nodes > (1 << 22)) return FMM_ERR_UNSUPPORTED;
  }
  node_rule->assign((size_t)nodes, 0);
  if (selection == FMM_SELECT_ROUND_ROBIN) {
    for (int64_t n = 0; n < nodes; ++n) (*node_rule)[(size_t)n] = (int)(n % 8);
    return FMM_OK;
  }
  if (selection == FMM_SELECT_RANDOM) {
    for (int64_t n = 0; n < nodes; ++n) (*node_rule)[(size_t)n] = (int)(splitmix64_at(seed, (uint64_t)n) >> 61);
    return FMM_OK;
  }
  if (selection != FMM_SELECT_MATRIX) return FMM_ERR_ARG;
  if (!block_max_a || !block_max_b) return FMM_ERR_ARG;
  std::vector<CanonRule> var(8);
  for (int v = 0; v < 8; ++v) var[v] = cg_variant(base, v);
  // Level by level: each node picks the variant with the smallest growth
  // estimate on its operand bounds (ties: the lowest index); its children's
  // bounds follow from the chosen variant's U and V.
  const int g = 1 << levels;
  Bounds a0, b0;
  a0.g = b0.g = g;
  a0.v.resize((size_t)g * g);
  b0.v.resize((size_t)g * g);
  for (int i = 0; i < g * g; ++i) {
    a0.v[i] = std::isfinite(block_max_a[i]) ? std::fabs((double)block_max_a[i]) : 0.0;
    b0.v[i] = std::isfinite(block_max_b[i]) ? std::fabs((double)block_max_b[i]) : 0.0;
  }
  std::vector<std::pair<Bounds, Bounds>> level{{a0, b0}};
  int64_t n = 0;
  for (int l = 0; l < levels; ++l) {
    std::vector<std::pair<Bounds, Bounds>> next;
    for (const auto& ab : level) {
      int best = 0;
      double best_cost = node_cost(var[0], ab.first, ab.second);
      for (int v = 1; v < 8; ++v) {
        const double cst = node_cost(var[v], ab.first, ab.second);
        if (cst < best_cost) {
          best_cost = cst;
          best = v;
        }
      }
      (*node_rule)[(size_t)n++] = best;
      if (l + 1 < levels)
        for (int r = 0; r < R; ++r)
          next.emplace_back(child_bounds(var[best], ab.first, r, true), child_bounds(var[best], ab.second, r, false));
    }
    level.swap(next);
  }
  return FMM_OK;
}

}  // namespace fmm
