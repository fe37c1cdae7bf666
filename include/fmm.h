/*
 * fmm.h -- C ABI of the GB300 (sm_103a) recursive fast matrix multiplication
 * library with power-of-two diagonal scaling.
 *
 * Method: Ballard, Benson, Druinsky, Lipshitz, Schwartz, "Improving the
 * numerical stability of fast matrix multiplication" (SIAM J. Matrix Anal.
 * Appl. 37(4), 2016).  C = A B with A (M x K) and B (K x N) computed by L
 * levels of bilinear rules [[U, V, W]] (Sec. 3, Eq. 3.1 / 3.2) and a
 * classical base case, optionally on the scaled operands of Sec. 6
 * (Algs. 1-3).
 *
 * Conventions (every entry point):
 *  - Matrices are row-major with a leading dimension (elements) >= the row
 *    length.  Device pointers are caller-owned CUDA device memory; the
 *    library never frees them.  Element data must be 16-byte aligned and
 *    leading dimensions multiples of 16 bytes for the vectorised paths;
 *    other layouts are accepted and take a slower element-wise path.
 *  - Calls that take a cudaStream_t (passed as void*, NULL = legacy default
 *    stream) are asynchronous: host-detectable errors return at once and
 *    launch nothing; errors the device detects (a bounded wait that ran out,
 *    a non-finite input to a scaling step) are recorded in a device status
 *    word that fmm_sync_status() reads and clears.
 *  - Exponent vectors are int32 device arrays: D_A = diag(2^eA) (length M),
 *    D = diag(2^d) (length K), D_B = diag(2^eB) (length N); any may be NULL
 *    (= all zeros).  The scaled operands A' = 2^-eA A 2^d and
 *    B' = 2^-d B 2^-eB are exact; fmm_multiply applies them while it
 *    forms the operand combinations and multiplies C by 2^(eA+eB) when it
 *    forms the output.
 *  - Every wait inside a kernel is bounded: FMM_WAIT_TIMEOUT_NS in the
 *    environment (read once per process; default 2 s) limits each one;
 *    past it the kernel stops cleanly and flags FMM_ERR_DEVICE_TIMEOUT.
 *    FMM_TEST_STALL=1 makes the tensor-core multiply wait once on a barrier
 *    that nothing arrives at, so that tests can exercise that path.
 *  - Device code needs sm_103a and the CUDA driver's tensor-map encoder.
 *  - Thread safety: plans are immutable after creation and may be used from
 *    several host threads; calls on one stream execute in order.
 */
#ifndef FMM_H_
#define FMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FMM_OK = 0,
  FMM_ERR_ARG = 1,            /* NULL pointer, negative size, bad enum      */
  FMM_ERR_NOT_MATMUL = 2,     /* a rule violates the Brent equations        */
  FMM_ERR_SHAPE = 3,          /* leading dimension too small, size limits   */
  FMM_ERR_ALIGN = 4,          /* reserved                                   */
  FMM_ERR_DTYPE = 5,          /* unsupported dtype / leaf-format pairing    */
  FMM_ERR_WORKSPACE = 6,      /* workspace missing or too small             */
  FMM_ERR_CUDA = 7,           /* a CUDA runtime call failed                 */
  FMM_ERR_DEVICE_TIMEOUT = 8, /* a kernel's bounded wait ran out            */
  FMM_ERR_NONFINITE = 9,      /* Inf/NaN met by a scaling step              */
  FMM_ERR_UNSUPPORTED = 10    /* plan shape outside what the kernels handle */
} fmm_status;

/* Single-index order of the entries of a base-case operand (Sec. 3.1). */
enum { FMM_ORDER_ROW = 0, FMM_ORDER_COL = 1 };

/* Element types of A and B in device memory. */
enum { FMM_DT_F32 = 0, FMM_DT_BF16 = 1, FMM_DT_F16 = 2 };

/* Leaf-product formats.  S_r and T_r are always formed in FP32; the leaf
 * rounds them to this format and multiplies on the tensor cores with FP32
 * accumulation.  BF16X3 splits x = hi + lo (hi = rn_bf16(x),
 * lo = rn_bf16(x - hi)) and sums hi*hi' + hi*lo' + lo*hi'.  E4M3B128: OCP
 * FP8 E4M3 with a power-of-two scale per 128-block along K (per row of S_r,
 * per column of T_r): s = e(block max) - 8, at least -127 (the scale is a
 * UE8M0 number), so the block's largest magnitude scales into [128, 256),
 * then round to nearest even; the leaf product sums 2^(sa + sb) times each
 * block's E4M3 products in FP32, the tensor core applying the scales
 * (block-scaled MMA; FMM_FP8_FOLD=1 in the environment, read once, folds
 * each block's product in the epilogue instead).  Pass schedule only. */
enum { FMM_LEAF_BF16 = 0, FMM_LEAF_F16 = 1, FMM_LEAF_BF16X3 = 2, FMM_LEAF_E4M3B128 = 3 };

/*
 * One base-case rule <m0, k0, n0; r> = [[U, V, W]] (Sec. 3.1, Eq. 3.1):
 *   C_k = sum_r W[k,r] M_r,  M_r = S_r T_r,
 *   S_r = sum_i U[i,r] A_i,  T_r = sum_j V[j,r] B_j.
 * U is (m0*k0) x r, V is (k0*n0) x r, W is (m0*n0) x r, each a host array
 * stored row-major (entry (i, r) at [i*r_count + r]).  order_a/b/c give how
 * the single index i (j, k) enumerates the entries of the m0 x k0 block of A
 * (of B, of C): FMM_ORDER_ROW or FMM_ORDER_COL.  The paper states A, B
 * column-major and C row-major (Sec. 3.1); its Strassen table (App. A)
 * needs A, B row-major and C column-major.  The arrays are copied by
 * fmm_plan; the caller keeps ownership.
 */
typedef struct {
  int m0, k0, n0, r;
  const double* U;
  const double* V;
  const double* W;
  int order_a, order_b, order_c;
} fmm_rule;

typedef struct fmm_plan_s* fmm_plan_t;

/*
 * Build a uniform non-stationary plan (Sec. 3.3; stationary when all levels
 * repeat one rule, Sec. 3.2): rules[l] is used at recursion level l+1,
 * l = 0..levels-1, and the classical algorithm at the leaves.  levels = 0 is
 * the classical product.  Every rule is checked against the Brent equations
 * (FMM_ERR_NOT_MATMUL on failure) and the levels are flattened into R^L
 * leaf descriptors (Eq. 4.4): leaf (r_1..r_L) multiplies
 *   S = sum prod_l U[i_l, r_l] A_(i_1..i_L),  T likewise with V,
 * and adds prod_l W[k_l, r_l] times its product into C block (k_1..k_L).
 * leaf_format is FMM_LEAF_*.  *out owns host and device memory; release it
 * with fmm_plan_destroy.  Uses the current CUDA device.
 */
fmm_status fmm_plan(fmm_plan_t* out, int levels, const fmm_rule* rules, int leaf_format);

/*
 * Build a non-uniform plan (Sec. 3.4): every node of the recursion tree
 * takes its own rule.  rules[0..nrules-1] is a table of distinct rules
 * (each checked against the Brent equations, FMM_ERR_NOT_MATMUL on
 * failure); node_rule[0..nnodes-1] gives each internal node's index into
 * that table, level by level from the root, and within a level in the order
 * of the parents and then of the parent's product index r = 0..R-1.  So
 * node_rule[0] is the root, the next R_root entries its children, and so on
 * down to level `levels`; below that every product is classical.  All nodes
 * of one level must share (m0, k0, n0), so that every root-to-leaf path
 * partitions A, B and C alike; their ranks R may differ.  FMM_ERR_ARG when
 * nnodes does not match the tree the ranks define, an index is out of range
 * or the dimensions of a level differ.  Leaves are flattened in depth-first
 * order (product r = 0..R-1 at every node), which for a tree with one rule
 * per level is the order fmm_plan uses.  fmm_plan_info then reports
 * max_k delta_k in place of sum Q and max_k xi_k in place of prod E (the
 * componentwise quantities of Sec. 4.5; they reduce to sum Q and prod E for
 * uniform plans), so fmm_plan_bound gives the bound of Sec. 4.5.  Scaling
 * between recursive steps needs every level's ranks equal (else
 * FMM_ERR_UNSUPPORTED).  The caller keeps ownership of rules and node_rule.
 */
fmm_status fmm_plan_tree(fmm_plan_t* out, int nrules, const fmm_rule* rules, int levels, int64_t nnodes,
                         const int32_t* node_rule, int leaf_format);

fmm_status fmm_plan_destroy(fmm_plan_t plan);

/*
 * Rule algebra.  Each call derives a new base-case rule from given ones,
 * checks the inputs and the result against the Brent equations
 * (FMM_ERR_NOT_MATMUL on failure) and writes the result's tables into the
 * caller's arrays U, V, W (row-major tables, sizes below), with out->U/V/W
 * pointing at them and all three entry orders FMM_ORDER_ROW.  Host only;
 * nothing is kept by the library.
 *
 * fmm_rule_rotate: the cyclic rotation of a <m0,k0,n0;r> rule into a
 *   <n0,m0,k0;r> rule (App. A-B: the matrix-multiplication tensor
 *   sum a_ik b_kj c_ij is invariant when its factors are cycled; the new A
 *   is C transposed, the new B is A, the new C is B transposed).  U holds
 *   n0*m0*r, V m0*k0*r, W n0*k0*r doubles.
 * fmm_rule_compose: two recursion steps as one rule (Eq. 4.4 with L = 2):
 *   the <m1 m2, k1 k2, n1 n2; r1 r2> rule whose product r1*r2_count + r2
 *   has coefficients X1[(p1,q1), r1] X2[(p2,q2), r2] at the composite entry
 *   (p1 m2 + p2, q1 k2 + q2).  FMM_ERR_UNSUPPORTED above 64 per dimension
 *   or 4096 products.  U holds m1 m2 k1 k2 r1 r2 doubles, and so on.
 * fmm_rule_transform: [[XU U, XV V, XW W]] (Sec. 3.4), XU (m0 k0 square),
 *   XV (k0 n0), XW (m0 n0) row-major, applied in the input rule's own
 *   entry orders; the arrays are the size of the input's.
 * fmm_rule_permute: the rule applied to A, B blocks whose indices are
 *   relabelled by the permutations perm_i (m0 entries), perm_k (k0),
 *   perm_j (n0) -- U'[(i,k)] = U[(perm_i[i], perm_k[k])],
 *   V'[(k,j)] = V[(perm_k[k], perm_j[j])], W'[(i,j)] = W[(perm_i[i],
 *   perm_j[j])] -- which computes the same product (the D'Alberto variant
 *   of Sec. 3.4 exchanges the j blocks); FMM_ERR_ARG when a perm_* is not a
 *   permutation.  Arrays the size of the input's.
 */
fmm_status fmm_rule_rotate(const fmm_rule* in, double* U, double* V, double* W, fmm_rule* out);
fmm_status fmm_rule_compose(const fmm_rule* outer, const fmm_rule* inner, double* U, double* V, double* W,
                            fmm_rule* out);
fmm_status fmm_rule_transform(const fmm_rule* in, const double* XU, const double* XV, const double* XW,
                              double* U, double* V, double* W, fmm_rule* out);
fmm_status fmm_rule_permute(const fmm_rule* in, const int32_t* perm_i, const int32_t* perm_k,
                            const int32_t* perm_j, double* U, double* V, double* W, fmm_rule* out);

/*
 * The eight Castrapel-Gustafson variants of a <2,2,2> rule (Sec. 3.4):
 *   [[(P^x (x) P^y) U, (P^z (x) P^x) V, (P^y (x) P^z) W]],  x, y, z in {1, 2},
 * P the 2 x 2 exchange, read in the paper's entry order (A, B column-major,
 * C row-major), where the factors exchange the k blocks (P^x), the i
 * blocks (P^y) and the j blocks (P^z); P^2 = I.  Variant v = 0..7 takes
 * x = 1 when bit 1 of v is set, y = 1 when bit 0 is set, z = 1 when bit 2
 * is set (else 2), so v = 0 is the rule itself.
 *
 * fmm_plan_variants builds the non-uniform plan of `levels` levels whose
 * every node runs one variant of `base`, chosen per node (the paper lists
 * random, round-robin and matrix-dependent selection without fixing them;
 * these are the library's definitions):
 *   FMM_SELECT_RANDOM: node n (level order, the node order of
 *     fmm_plan_tree) takes the top three bits of SplitMix64 output n of
 *     stream `seed` (z = seed + (n+1) 0x9E3779B97F4A7C15, then the
 *     generator's two xor-shift-multiply rounds and final xor-shift);
 *   FMM_SELECT_ROUND_ROBIN: node n takes variant n mod 8;
 *   FMM_SELECT_MATRIX: from the block max-abs values of A and B on the
 *     plan's finest grid (block_max_a, block_max_b: 2^levels x 2^levels,
 *     row-major, as fmm_block_max writes them), level by level: each node
 *     takes the variant minimising max_k sum_r |W_kr| (sum_i |U_ir| a_i)
 *     (sum_j |V_jr| b_j), the one-level growth factor of the proof of
 *     Theorem 4.1 on its own operands, with a_i, b_j bounds on the max-abs
 *     of its operands' quadrants (ties: the lowest v); the bounds of the
 *     operands S_r, T_r of its children follow by the triangle inequality
 *     from the chosen U and V (sums in ascending index order, in double).
 * block_max_* are host arrays, read only for FMM_SELECT_MATRIX (else
 * may be NULL).  chosen (nullable, host, 1 + R + ... + R^(levels-1)
 * entries) receives each node's variant.  FMM_ERR_UNSUPPORTED unless base
 * is <2,2,2>; otherwise as fmm_plan_tree.
 */
enum { FMM_SELECT_RANDOM = 0, FMM_SELECT_ROUND_ROBIN = 1, FMM_SELECT_MATRIX = 2 };
fmm_status fmm_plan_variants(fmm_plan_t* out, const fmm_rule* base, int levels, int selection, uint64_t seed,
                             const float* block_max_a, const float* block_max_b, int32_t* chosen,
                             int leaf_format);

/*
 * Block max-abs of a row-major matrix X (rows x cols, ld, element type
 * dtype, device memory) cut into nrb x ncb blocks of ceil(rows/nrb) x
 * ceil(cols/ncb) elements, as a plan partitions its operands (Sec. 3.2;
 * missing elements of ragged edge blocks count as zero): out[p*ncb + q] =
 * max |X| over block (p, q), float32, device memory.  Inf/NaN entries are
 * skipped and flagged in the status word (FMM_ERR_NONFINITE from
 * fmm_sync_status).  nrb, ncb in 1..64.  Asynchronous on the stream.
 */
fmm_status fmm_block_max(const void* X, int dtype, int64_t rows, int64_t cols, int64_t ld, int nrb, int ncb,
                         float* out, void* stream);

/*
 * Principal quantities of the plan (Sec. 4.1, Theorem 4.2): sum over levels
 * of Q (Def. 4.1), product of E (Def. 4.2), number of leaves R^L,
 * nnz of the flattened [[U, V, W]], and the products of m0, k0, n0 over the
 * levels (the padding granules).  Any output pointer may be NULL.
 */
fmm_status fmm_plan_info(fmm_plan_t plan, double* q_sum, double* e_prod, int64_t* leaves,
                         int64_t* nnz, int64_t* pm, int64_t* pk, int64_t* pn);

/* Tables fmm_plan_flatten reads back. */
enum { FMM_TABLE_LEAVES = 0, FMM_TABLE_LISTS = 1, FMM_TABLE_GATHER = 2 };

/*
 * The plan's flattened rule [[U^(L), V^(L), W^(L)]] (Eq. 4.4; for a tree,
 * Sec. 3.4, each leaf flattened along its own root-to-leaf path), read back
 * from one of the tables the kernels execute, so that a caller can check
 * them against its own derivation or export the algorithm.  Dense,
 * row-major, in host memory the caller provides (sizes from fmm_plan_info):
 * U is (pm pk) x leaves, V (pk pn) x leaves, W (pm pn) x leaves, entry
 * (i, r) at [i * leaves + r], with i = p pk + q for block (p, q) of A's
 * pm x pk block grid (B's and C's grids likewise).  first (optional, int32,
 * W's shape) is 1 where leaf r is the first in leaf order to add into C
 * block k (there the fused epilogue stores instead of adding), else 0.
 * table: FMM_TABLE_LEAVES = the per-leaf descriptors the tensor-core kernels
 * read; FMM_TABLE_LISTS = the per-side term lists of the combination and
 * output passes; FMM_TABLE_GATHER = the per-C-block lists of the gather
 * output pass (W and first only, U and V are not written;
 * FMM_ERR_UNSUPPORTED when pm pn > 2^20, where the plan carries none).  Any
 * of U, V, W, first may be NULL.  Coefficients are the float values the
 * kernels multiply by.  Host only (no device access, no allocation); the
 * dense tables grow as blocks x leaves, so this is meant for plans of up
 * to some thousands of leaves.  FMM_ERR_ARG for a NULL plan or an unknown
 * table.
 */
fmm_status fmm_plan_flatten(fmm_plan_t plan, int table, double* U, double* V, double* W,
                            int32_t* first);

/*
 * First-order bound of Theorem 4.2 for this plan and a K-dimension:
 *   (Kl + sum Q)(Kl) (prod E) normA normB eps,  Kl = ceil(K / prod k0).
 */
fmm_status fmm_plan_bound(fmm_plan_t plan, int64_t K, double normA, double normB, double eps,
                          double* bound);

/*
 * O step of Alg. 3 (Alg. 1 when d_in is NULL) in power-of-two form:
 *   eA[i] = e(max_k |A_ik| 2^d_k),   eB[j] = e(max_k 2^-d_k |B_kj|),
 * e(x) the frexp exponent (x = f 2^e, 1/2 <= f < 1), 0 for an all-zero
 * row / column.  The scaled operands 2^-eA A 2^d and 2^-d B 2^-eB then have
 * row (column) maxima in [1/2, 1) (Prop. 6.1).  A is M x K (lda), B is
 * K x N (ldb), both of element type dtype (FMM_DT_*).  d_in: length K or
 * NULL.  eA (length M) and eB (length N) are overwritten.  Inf/NaN in A or
 * B sets FMM_ERR_NONFINITE in the device status word.
 */
fmm_status fmm_scale_outside(const void* A, const void* B, int dtype, int64_t M, int64_t K,
                             int64_t N, int64_t lda, int64_t ldb, const int32_t* d_in,
                             int32_t* eA, int32_t* eB, void* stream);

/*
 * I step of Alg. 3 (Alg. 2 when eA, eB are NULL), Eq. 6.6 in power-of-two
 * form, on the operands currently scaled by eA and eB:
 *   d[k] = floor((e(max_j |B_kj| 2^-eB_j) - e(max_i 2^-eA_i |A_ik|)) / 2),
 * 0 when either maximum is zero.  The result replaces any previous d (the
 * cumulative inside scale of Alg. 3 equals this value, because previous
 * inside exponents cancel out of the ratio).  d has length K.
 */
fmm_status fmm_scale_inside(const void* A, const void* B, int dtype, int64_t M, int64_t K,
                            int64_t N, int64_t lda, int64_t ldb, const int32_t* eA,
                            const int32_t* eB, int32_t* d, void* stream);

/*
 * Alg. 3 with a fixed step sequence: steps is a string over {'O','I'}
 * ("O" = Alg. 1, "I" = Alg. 2, "OI" = outside then inside, "OIOI" = twice
 * repeated).  eA, d, eB are zeroed first and then updated by each step.
 */
fmm_status fmm_scale(const char* steps, const void* A, const void* B, int dtype, int64_t M,
                     int64_t K, int64_t N, int64_t lda, int64_t ldb, int32_t* eA, int32_t* d,
                     int32_t* eB, void* stream);

/*
 * Adaptive Alg. 3 (Sec. 6.3): O and I steps alternate, starting with an O
 * step (first_inside = 0) or an I step (first_inside = 1), for at most
 * max_steps steps.  Each step after the first O step is tested on the
 * power-of-two factors it applies, 2^(new - old exponent): an O step
 * passes when every row factor of A and column factor of B is at least
 * (1 + tau)^(-1/2), an I step when every inside factor lies in
 * [(1 + tau)^(-1/4), (1 + tau)^(1/4)].  The iteration stops after the first
 * step that passes, keeping its result; the theorem of Sec. 6.3 puts the
 * real-valued scales within relative distance tau of their limit there.
 * With tau < 3 only factors of 1 pass the I test and only factors >= 1 the
 * O test, so the power-of-two iteration stops at a fixed point.  tau > 0.
 * eA (M), d (K), eB (N) receive the exponents, as fmm_scale.  steps_taken
 * (device int32, may be NULL) receives the number of steps applied.  The
 * stop is decided on the device: all max_steps steps are launched and
 * those after the stop return at once, so the host does not wait and the
 * call can be captured in a CUDA graph.  ws: device workspace of at least
 * 4 (M + K + N + 64) bytes, 16-byte aligned (FMM_ERR_WORKSPACE otherwise).
 */
fmm_status fmm_scale_adaptive(const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                              int64_t lda, int64_t ldb, double tau, int max_steps, int first_inside,
                              int32_t* eA, int32_t* d, int32_t* eB, int32_t* steps_taken, void* ws,
                              size_t ws_bytes, void* stream);

/*
 * Where a multiply forms the operand combinations S_r = sum u A_i and
 * T_r = sum v B_j of Eq. 4.4 (the products and the output combination are
 * the same in both; so are the sums, in FP32 in index order, and their
 * rounding to the leaf format, hence the results):
 *   FMM_SCHEDULE_LOAD_STAGE  in the load stage of the multiply kernel: the
 *     term tiles are staged in shared memory and summed by producer warps
 *     into the tensor-core operand tiles; workspace only for prepared
 *     operand copies;
 *   FMM_SCHEDULE_PASS        by a bandwidth-bound combination pass that
 *     writes every S_r and T_r once, in the leaf format, into the workspace
 *     (R^L leaf blocks per operand, two planes for the hi+lo split); the
 *     multiply kernel then streams them with bulk tensor copies;
 *   FMM_SCHEDULE_AUTO        (default) the pass schedule when the given
 *     workspace holds it, else the load-stage schedule.
 * Under the pass schedule the output combination C_k += sum w M_r (Eq. 4.4,
 * third line) runs either in the multiply kernel's epilogue (one CTA per
 * output tile position visits every leaf) or, when one leaf's tiles are too
 * few to occupy the GPU (deep recursion, small products), over stored leaf
 * products: every (leaf, tile) pair is a unit of work, the epilogue stores
 * M_r in the workspace and a bandwidth-bound pass forms C.  Both give the
 * same result (the same operations per element, in leaf order).
 * FMM_SCHEDULE_PASS (and AUTO) use stored products when the workspace
 * holds them (measured faster on GB300 at every size tried);
 * FMM_SCHEDULE_PASS_EPILOGUE and FMM_SCHEDULE_PASS_PRODUCTS force one form.
 * Stored products need a plan of more than one leaf and at most 96 C
 * blocks; otherwise the epilogue form runs.
 *   FMM_SCHEDULE_PASS_ACCUMULATE  the pass schedule with every (leaf, tile)
 *     unit adding its W-weighted, unscaled terms into C (zeroed first) by
 *     atomic FP32 additions in the multiply kernel's epilogue: no stored
 *     products, no output pass.  The order in which an element's terms
 *     arrive varies from run to run, so results may differ in the last
 *     bits between runs (each is within the same error bound).  Taken by
 *     the CTA-pair kernel (leaf blocks of at least 256 x 256, 16-bit
 *     leaves); other products run as FMM_SCHEDULE_PASS.
 */
#define FMM_SCHEDULE_AUTO 0
#define FMM_SCHEDULE_LOAD_STAGE 1
#define FMM_SCHEDULE_PASS 2
#define FMM_SCHEDULE_PASS_EPILOGUE 3
#define FMM_SCHEDULE_PASS_PRODUCTS 4
#define FMM_SCHEDULE_PASS_ACCUMULATE 5

/* Set the plan's schedule (FMM_SCHEDULE_*); FMM_ERR_ARG for other values.
 * The gradient products of fmm_multiply_backward follow it. */
fmm_status fmm_plan_set_schedule(fmm_plan_t plan, int schedule);

/*
 * Scaling between recursive steps (opt-in; plans of two or more levels;
 * the paper applies Algs. 1-3 to the whole product only, so this is an
 * extension: each sub-product of a recursive step is itself a matrix
 * product, and it is scaled as one).  After the first level's operand sums
 * S_r, T_r are formed (in FP32, in index order), each pair is inside-scaled
 * as its own product A B -- Alg. 2 in power-of-two form,
 *   d^(r)_k = floor((e(max_j |T_r[k, j]|) - e(max_i |S_r[i, k]|)) / 2),
 * 0 where either side is zero -- S_r <- S_r 2^d, T_r <- 2^-d T_r, before the
 * lower levels combine them.  The scale cancels exactly in every product,
 * so only rounding changes.  Forward products under the pass schedule only:
 * fmm_multiply returns FMM_ERR_UNSUPPORTED under the load-stage schedule,
 * fmm_multiply_backward and fmm_multiply_noalloc ignore it, batches reject
 * it.  enable = 0 turns it off.  A no-op for plans of fewer than two levels.
 */
fmm_status fmm_plan_set_between_scaling(fmm_plan_t plan, int enable);

/*
 * Workspace bytes fmm_multiply / fmm_multiply_backward need for this plan
 * and shape (an upper bound over input types).  The fused kernel reads its
 * operands through tensor-memory-access copies of whole 128 x 64 tiles; an
 * operand whose leaf blocks are not whole tiles, whose rows are not 16-byte
 * aligned, that is scaled (exponent vectors given) or fp16 is first written,
 * by one bandwidth-bound pass, as a blocked, zero-padded, scaled copy into
 * the workspace.  Calls whose operands need no copy may pass NULL / 0.
 * Under the AUTO and PASS schedules the size also covers the combined
 * operands of the pass schedule (see fmm_plan_set_schedule).
 */
fmm_status fmm_workspace_size(fmm_plan_t plan, int64_t M, int64_t K, int64_t N, size_t* bytes);

/*
 * C = A B by the plan's fast algorithm (Eq. 3.2), on the scaled operands
 * when exponents are given (Algs. 1-3: C = D_A (A' B') D_B).  A: M x K
 * (lda), B: K x N (ldb), element type in_dtype; C: M x N float32 (ldc),
 * overwritten.  M, K, N are zero-padded internally up to multiples of the
 * plan's granules (Sec. 3.2).  What runs depends on the plan's schedule
 * (fmm_plan_set_schedule) and the workspace given:
 *  - the pass schedule (the default whenever ws holds fmm_workspace_size
 *    bytes): one launch forms every S_r and T_r (both operands, scaling
 *    applied) into the workspace; one tensor-core launch forms the leaf
 *    products (on CTA pairs with 256 x 256 tiles when the leaf blocks are
 *    at least 256 x 256, else one CTA per 128 x 256 tile) and stores them;
 *    one output pass forms C = sum w M_r, unscaled -- three launches (plus
 *    the between-steps exponent kernels when that scaling is on); a
 *    single-leaf plan adds its product into C in the multiply epilogue;
 *    with 16-bit leaves on CTA pairs, where the multiply is compute-bound
 *    (leaf K >= 2048, at most 16 leaves and 16 C blocks, each half of the
 *    tile rows filling the GPU for 5 waves or more), it runs as two
 *    launches over the tile-row halves, and the first half's output pass
 *    runs on a library-owned side stream beside the second half's
 *    multiply, joined back to the caller's stream by events (FMM_OVERLAP=0
 *    in the environment, read once, keeps one launch); E4M3 leaves always
 *    take the pass schedule, with their own combination pass (the E4M3
 *    bytes and the per-block scales) and the block-scaled multiply;
 *  - the load-stage schedule: one launch forms S_r, T_r in the multiply
 *    kernel's load stage and adds W-weighted products into C in its
 *    epilogue (operands needing a prepared copy get one bandwidth pass).
 * Results are deterministic (each C element summed by one thread in leaf
 * order) except under FMM_SCHEDULE_PASS_ACCUMULATE.  ws/ws_bytes: device
 * workspace, 256-byte aligned, of fmm_workspace_size bytes (NULL / 0 runs
 * the load-stage schedule when no operand needs a copy); FMM_ERR_WORKSPACE
 * if a needed workspace is missing or too small.
 */
fmm_status fmm_multiply(fmm_plan_t plan, const void* A, int64_t lda, const void* B, int64_t ldb,
                        float* C, int64_t ldc, int64_t M, int64_t K, int64_t N, int in_dtype,
                        const int32_t* eA, const int32_t* d, const int32_t* eB, void* ws,
                        size_t ws_bytes, void* stream);

/* Size of the static scratch array fmm_multiply_noalloc works in. */
#define FMM_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/*
 * fmm_multiply without a caller-supplied workspace and without allocating
 * anything.  The paper has no counterpart: this is a library convenience.
 *
 * Who needs it: code that must not call cudaMalloc (or any allocator) on
 * the device -- for instance a caller running under a memory pool or arena
 * that owns all device memory, a plugin inside a host framework that does
 * not hand out scratch buffers, or code on a latency-critical path where an
 * allocation could synchronise the device.  Such a caller passes only its
 * inputs and output; the scratch (the plan's leaf table and the prepared
 * operand copies described under fmm_workspace_size) lives in one array of
 * FMM_NOALLOC_SCRATCH_BYTES bytes that the library declares in device
 * memory.  Every GPU that loads the library holds that array until the
 * process exits.
 *
 * Arguments, layouts and results are those of fmm_multiply (scaling
 * between recursive steps is not applied).  Returns FMM_ERR_WORKSPACE,
 * before touching the device, when the leaf table plus the workspace of
 * the path the call would take exceeds FMM_NOALLOC_SCRATCH_BYTES: the pass
 * schedule's combined operands and stored products for E4M3 leaves and
 * the forced pass schedules, the prepared operand copies (fp32 upper
 * bound) under FMM_SCHEDULE_LOAD_STAGE, the smaller of the two under
 * FMM_SCHEDULE_AUTO; fmm_last_error() then says how many bytes the problem
 * needs.  About n <= 2000 for a square fp32 product at one level.
 *
 * The first call on a device looks up the array's device address (once
 * per device); make that first call before any stream capture begins.
 * Each call copies the plan's tables into the array with small kernel
 * launches that carry the data in their arguments (no copy from host
 * memory, nothing for the host to wait on).  Nothing in the array needs to
 * start at zero: each call writes the tables and every element of the
 * operands it forms (padding included) before a kernel reads them.  All
 * calls share the one array, so calls whose work overlaps on the GPU
 * (different streams, or threads without ordering) race on it and give
 * wrong results; order them on one stream.
 */
fmm_status fmm_multiply_noalloc(fmm_plan_t plan, const void* A, int64_t lda, const void* B,
                                int64_t ldb, float* C, int64_t ldc, int64_t M, int64_t K,
                                int64_t N, int in_dtype, const int32_t* eA, const int32_t* d,
                                const int32_t* eB, void* stream);

/*
 * Batches (the batched multiply of the call list: fmm_batch_create /
 * fmm_batch_run / fmm_batch_destroy together are fmm_multiply_batched,
 * split so that all host work and table uploads happen once and a run only
 * launches): many independent products of uneven shapes, each with its own
 * plan (rule, recursion depth), run as one fixed sequence of launches over
 * all of them -- the batched scaling reductions, one combination pass, ONE
 * persistent tensor-core launch over every product's (leaf, tile) work
 * units, one output pass -- so a whole batch costs about nine launches.
 * fmm_batch_create does all host work and every allocation-free layout
 * decision once: it checks the problems, lays out the per-product exponent
 * vectors, combined operands and stored leaf products, and the launch
 * tables, in the caller's workspace (ws, 256-byte aligned, of
 * fmm_batch_workspace_size bytes), and copies the tables there
 * (synchronously).  fmm_batch_run then only launches kernels on the stream,
 * with no host synchronisation or allocation, so it can be captured in a
 * CUDA graph and replayed; each replay recomputes every C from the current
 * contents of the A and B buffers.
 *
 * All plans of a batch must share their leaf format, and each must have at
 * most 96 C blocks (pm x pn); every M, K, N must be positive.  A and B have
 * element type in_dtype; steps is "" (no scaling), "O", "I" or "OI" (Alg. 3
 * steps starting from no scaling, as fmm_scale; the exponents live in the
 * workspace).  The plans, the batch and the workspace must outlive every run.
 */
typedef struct {
  fmm_plan_t plan;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
  int64_t M, K, N;
} fmm_problem;

typedef struct fmm_batch_s* fmm_batch_t;

fmm_status fmm_batch_workspace_size(const fmm_problem* problems, int count, int in_dtype,
                                    const char* steps, size_t* bytes);
fmm_status fmm_batch_create(fmm_batch_t* out, const fmm_problem* problems, int count, int in_dtype,
                            const char* steps, void* ws, size_t ws_bytes);
fmm_status fmm_batch_run(fmm_batch_t batch, void* stream);
fmm_status fmm_batch_destroy(fmm_batch_t batch);

/*
 * Split a batch over `parts` GPUs (one process per GPU, each running its
 * share as a batch of its own: independent products need no exchange):
 * longest-processing-time order by the classical flop count 2 M K N (ties
 * by index), each product to the part with the least assigned flops so far
 * (ties: the lowest part), so the largest share is within 4/3 of the best
 * possible.  M, K, N: host arrays of `count` sizes; part_of (host, count
 * entries) receives each product's part.  Host only; the same inputs give
 * the same assignment on every process.
 */
fmm_status fmm_batch_partition(const int64_t* M, const int64_t* K, const int64_t* N, int count, int parts,
                               int32_t* part_of);

/*
 * Gradients of C = A B for a given dC (M x N, float32, lddc):
 *   dA = dC B^T (M x K, float32, ldda),  dB = A^T dC (K x N, float32, lddb),
 * each by a fast algorithm derived from the plan's rules through the cyclic
 * symmetry of the matrix-multiplication tensor (the rule transforms of
 * Sec. 5.3 and App. A-C): dA uses [[W, V^T, U]] (an <m0,n0,k0> rule), dB
 * uses [[U^T, W, V]] (a <k0,m0,n0> rule), where ^T re-indexes the operand's
 * entries by transposition.  dA or dB may be NULL to skip it.  A and B have
 * element type in_dtype.  ws/ws_bytes: device workspace as for fmm_multiply
 * (fmm_workspace_size covers both passes; the two products run one after
 * the other and reuse it).
 */
fmm_status fmm_multiply_backward(fmm_plan_t plan, const float* dC, int64_t lddc, const void* A,
                                 int64_t lda, const void* B, int64_t ldb, float* dA,
                                 int64_t ldda, float* dB, int64_t lddb, int64_t M, int64_t K,
                                 int64_t N, int in_dtype, void* ws, size_t ws_bytes, void* stream);

/* Gradients fmm_plan_gradient returns the plan of. */
enum { FMM_GRAD_A = 0, FMM_GRAD_B = 1 };

/*
 * The plan fmm_multiply_backward runs for one gradient, as a plan of its
 * own (for inspection with fmm_plan_info / fmm_plan_flatten, or to run a
 * gradient product through fmm_multiply): FMM_GRAD_A gives the
 * <pm, pn, pk> plan of dA = dC B^T whose levels (or tree nodes) use
 * [[W, V^T, U]], FMM_GRAD_B the <pk, pm, pn> plan of dB = A^T dC with
 * [[U^T, W, V]]; a tree keeps its shape, every node's rule transformed;
 * the leaf format and schedule are the plan's.  *out is a new plan owned
 * by the caller (fmm_plan_destroy).  Host only.  FMM_ERR_ARG for a NULL
 * plan or out, or an unknown `which`.
 */
fmm_status fmm_plan_gradient(fmm_plan_t plan, int which, fmm_plan_t* out);

/*
 * Host-memory pipeline (not from the paper: the paper's products live in
 * one memory).  For a stream of products of one shape whose operands and
 * results are in host memory, fmm_host_create sets up `depth` (1..4) slots
 * of device memory (A, B, C, the exponent vectors) plus one workspace, and
 * four streams: copy-in of A, copy-in of B, compute, copy-out.  fmm_host_submit enqueues one
 * product and returns without waiting: the host->device copies of A (M x K,
 * lda) and B (K x N, ldb) into the next slot, then -- once they are in --
 * the scaling steps (`steps` as in fmm_scale, "" for none) and
 * fmm_multiply, then the device->host copy of C (M x N, ldc, float32).  A
 * slot is reused only after its previous product has been read and
 * written back, so with depth >= 2 the copies of one product overlap the
 * computation of its neighbours.  The caller must leave the host buffers of
 * a submission untouched until fmm_host_wait returns (or until `depth`
 * further submissions); page-locked host memory lets the copies run
 * asynchronously, pageable memory works but serialises them.  dtype is
 * FMM_DT_*.  The pipeline keeps a reference to the plan, which must
 * outlive it.  Errors: FMM_ERR_ARG (bad sizes, depth, steps), FMM_ERR_CUDA.
 */
typedef struct fmm_host_s* fmm_host_t;
fmm_status fmm_host_create(fmm_host_t* out, fmm_plan_t plan, int64_t M, int64_t K, int64_t N, int dtype,
                           const char* steps, int depth);
fmm_status fmm_host_submit(fmm_host_t h, const void* hA, int64_t lda, const void* hB, int64_t ldb, float* hC,
                           int64_t ldc);
/* Wait until every submitted product is back in host memory; returns the
 * first error any of them met (the device status word included). */
fmm_status fmm_host_wait(fmm_host_t h);
fmm_status fmm_host_destroy(fmm_host_t h);

/*
 * Per-kernel timing, for measurement.  fmm_kernel_timing(1) starts
 * recording (discarding earlier records): every kernel the library launches
 * from then on is bracketed by two CUDA events recorded on its launching
 * stream; fmm_kernel_timing(0) stops recording.  Any other value in 2..31
 * records only the kinds whose bits it sets: 2 "scale" (scaling reductions
 * and fills), 4 "prepare" (operand copies of the load-stage schedule), 8
 * "combine" (the combination and output passes), 16 "multiply" (the
 * tensor-core kernels); FMM_ERR_ARG outside 0..31.  fmm_kernel_timing_read
 * waits for the recorded events and returns the summed device time (ms)
 * and the number of launches of one kind, or of all kinds when kind is NULL
 * or "".  The library's own work is unchanged, but an event between two
 * launches keeps the second from starting before the first ends (the
 * kernels otherwise overlap one's start with the other's end), and the
 * events add a few microseconds of host time per launch.
 */
fmm_status fmm_kernel_timing(int enable);
fmm_status fmm_kernel_timing_read(const char* kind, double* total_ms, int64_t* launches);

/*
 * Synchronise the stream, then read and clear the device status word.
 * Returns FMM_OK, FMM_ERR_DEVICE_TIMEOUT, FMM_ERR_NONFINITE or FMM_ERR_CUDA.
 */
fmm_status fmm_sync_status(void* stream);

/*
 * Text of the last CUDA runtime error a library call on this host thread
 * met, or of the last size rejection by fmm_multiply_noalloc (empty when
 * none); the pointer stays valid until the next library call on the
 * thread.
 */
const char* fmm_last_error(void);

/* Static English description of a status code. */
const char* fmm_status_string(fmm_status s);

/* Library version string. */
const char* fmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H_ */
