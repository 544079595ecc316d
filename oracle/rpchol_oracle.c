/*
 * FP64 CPU oracle for randomly pivoted Cholesky (Epperly, Tropp, Webber,
 * "Embrace rejection: Kernel matrix approximation by accelerated randomly
 * pivoted Cholesky", arXiv 2410.03969).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What is here, each written from the paper's text:
 *   - orc_philox4x32_10 / orc_u53: the counter-based random source.  The
 *     paper only says "Rand()" (Algorithm 1); the generator is Philox4x32-10
 *     from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 *     1, 2, 3" (SC'11), written from that description.
 *   - orc_kernel_entry: Gaussian (Eq. "gaussian", Sec. 1.2), Matern-5/2
 *     (Sec. 3.2), the l2-Laplace exp(-||x-y||/sigma), Matern-3/2 (named in
 *     the testbed of Sec. 4 without a formula; the textbook
 *     (1 + sqrt3 r/sigma) exp(-sqrt3 r/sigma) is taken) through direct
 *     differences sum_l (x_l - y_l)^2, as the paper's block experiments do
 *     (App. A.1, last paragraph), and the l1-Laplace
 *     exp(-sum_l |x_l - y_l| / sigma) (Eq. "l1_laplace", Sec. 1.2) through
 *     the sum of absolute differences.
 *   - orc_sample: one draw from the distribution w / sum(w) (Eq. 1.3 and
 *     the proposal step of Algorithm 2).
 *   - orc_reject_chol: RejectionSampleSubmatrix, Algorithm 1.
 *   - orc_rpc_plain: simple RPCholesky, Algorithm 6 (appendix).
 *   - orc_rpc_accel: accelerated RPCholesky, Algorithm 2, calling Algorithm 1.
 *   - orc_rpc_block: block RPCholesky, Algorithm 7 (appendix).
 *   - orc_rpqr_accel: accelerated randomly pivoted QR, Algorithm 5
 *     (appendix), on a dense rectangular matrix.
 *   - orc_rpc_lowmem: the low-memory form of Algorithm 2, Algorithm 3
 *     (Sec. 2.4): pivots and the k x k Cholesky factor of A(S,S) only.
 *   - orc_fixed_pivot_factor: Cholesky with a given pivot order; it gives the
 *     exact Nystrom approximation A(:,S) A(S,S)^+ A(S,:) of Sec. 2.1 so that
 *     a pivot list produced elsewhere can be re-evaluated in FP64.
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes of the repository):
 *   - random stream: Philox key = (seed low word, seed high word); the block
 *     for round r, proposal slot j, instance m uses counter (j, r, 0, m);
 *     words (w0,w1) give the proposal uniform, (w2,w3) the acceptance
 *     uniform.  Simple RPCholesky step i uses counter (0, i, 0, m), words
 *     (w0,w1), the same uniform as accelerated round i slot 0.
 *   - uniform from two words: ((w_a >> 5) * 2^26 + (w_b >> 6)) * 2^-53.
 *   - proposal map: W = sum of weights in index order, C_j the inclusive
 *     prefix sum in index order, pick min{ j : C_j > U*W }; if rounding
 *     leaves none, the largest j with w_j > 0.  Zero weights never chosen.
 *   - acceptance (Algorithm 1 test "u_i * Rand() < h_ii"): u_i is the weight
 *     d[s'_i] that proposal i was drawn with (the rejection-sampling box of
 *     Sec. 2.1 divides by the proposal weight); strict "<" in FP64.
 *   - reaching exactly k: Algorithm 1 stops as soon as the total rank is k;
 *     the remaining proposals of that round are ignored.
 *   - the diagonal u is clamped at zero after every round / step
 *     (Algorithm 2, last line), in both algorithms.
 *   - simple RPCholesky: F(:,i) = g / sqrt(g_s) with g_s taken from the
 *     freshly formed column (Algorithm 6).  If g_s <= 0 (only possible
 *     through rounding) the step adds no column, sets d[s] = 0 and moves on.
 *   - G = R L^{-*} (Algorithm 2, step 3) is solved row by row by forward
 *     substitution with the lower-triangular L.
 *
 * Floating point: everything in IEEE double; compiled with
 * -ffp-contract=off so that results do not depend on FMA contraction of the
 * host compiler (x86-64 and aarch64 give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Residual floor (the paper stops when the weights sum to 0, in exact
 * arithmetic): a residual weight at or below ORC_D_FLOOR (relative to the
 * largest diagonal entry, 1 for the kernels) is rounding noise on an
 * exhausted row; it is set to 0 together with the clamp at 0.  Without it
 * a numerically rank-deficient kernel matrix keeps a few weights near
 * 1e-16 whose recomputed Schur diagonals are far smaller, so Algorithm 1
 * rejects them round after round and the run never stops.                  */
#define ORC_D_FLOOR 1e-12

/* The floor for weights that start at d (times the largest of them).      */
static double orc_floor(const double* d, int64_t N)
{
    double m = 0.0;
    for (int64_t j = 0; j < N; ++j) m = d[j] > m ? d[j] : m;
    return ORC_D_FLOOR * m;
}

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

enum { ORC_GAUSSIAN = 0, ORC_LAPLACE_L2 = 1, ORC_MATERN52 = 2, ORC_MATERN32 = 3, ORC_LAPLACE_L1 = 4 };

static int orc_threads = 1;

int orc_set_threads(int n)
{
    orc_threads = n < 1 ? 1 : n;
#ifdef _OPENMP
    return orc_threads;
#else
    orc_threads = 1;
    return 1;
#endif
}

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11).  One round maps (c0,c1,c2,c3) with
 * key (k0,k1) through two 32x32->64 multiplications:
 *   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2
 *   c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
 * and the key is bumped by the Weyl constants between rounds.            */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* A uniform double in [0, 1 - 2^-53] from 27 + 26 random bits. */
double orc_u53(uint32_t a, uint32_t b)
{
    uint64_t hi = (uint64_t)(a >> 5);
    uint64_t lo = (uint64_t)(b >> 6);
    return (double)(hi * 67108864u + lo) * (1.0 / 9007199254740992.0);
}

/* The two uniforms of one Philox block: proposal (w0,w1), acceptance (w2,w3). */
void orc_uniform_pair(uint64_t seed, uint32_t slot, uint32_t round, uint32_t inst,
                      double* u_prop, double* u_acc)
{
    uint32_t ctr[4] = {slot, round, 0u, inst};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    if (u_prop) *u_prop = orc_u53(w[0], w[1]);
    if (u_acc) *u_acc = orc_u53(w[2], w[3]);
}

/* ---------------------------------------------------------------------- */
/* Kernel functions phi with kappa(x,x') = phi(q): q = ||x - x'||_2^2 for
 * the Euclidean kernels, q = ||x - x'||_1 for the l1-Laplace.             */
static double orc_phi_from_r2(int kind, double sigma, double r2)
{
    if (r2 < 0.0) r2 = 0.0;
    switch (kind) {
    case ORC_GAUSSIAN:
        return exp(-r2 / (2.0 * sigma * sigma));
    case ORC_LAPLACE_L2: {
        double r = sqrt(r2);
        return exp(-r / sigma);
    }
    case ORC_MATERN52: {
        double r = sqrt(r2);
        double t = sqrt(5.0) * r / sigma;
        return (1.0 + t + 5.0 * r2 / (3.0 * sigma * sigma)) * exp(-t);
    }
    case ORC_MATERN32: {
        double t = sqrt(3.0) * sqrt(r2) / sigma;
        return (1.0 + t) * exp(-t);
    }
    case ORC_LAPLACE_L1:
        return exp(-r2 / sigma);
    default:
        return NAN;
    }
}

double orc_phi(int kind, double sigma, double r2) { return orc_phi_from_r2(kind, sigma, r2); }

/* kappa(x_i, x_j) by direct differences; the diagonal is phi(0) = 1 exactly. */
static double orc_point_entry(int kind, double sigma, const float* X, int d, int64_t i, int64_t j)
{
    if (i == j) return 1.0;
    const float* xi = X + i * (int64_t)d;
    const float* xj = X + j * (int64_t)d;
    double q = 0.0;
    for (int l = 0; l < d; ++l) {
        double t = (double)xi[l] - (double)xj[l];
        q += kind == ORC_LAPLACE_L1 ? fabs(t) : t * t;
    }
    return orc_phi_from_r2(kind, sigma, q);
}

/* A matrix seen through the submatrix access model: either kernel entries
 * of points X (N x d, row-major, float) or an explicit dense psd matrix
 * (N x N, row-major, double) used by the tests.                           */
typedef struct {
    const float* X;
    int d;
    int kind;
    double sigma;
    const double* A;
    int64_t N;
} orc_matrix;

static double orc_entry(const orc_matrix* M, int64_t i, int64_t j)
{
    if (M->A) return M->A[i * M->N + j];
    return orc_point_entry(M->kind, M->sigma, M->X, M->d, i, j);
}

double orc_kernel_entry(int kind, double sigma, const float* X, int d, int64_t i, int64_t j)
{
    return orc_point_entry(kind, sigma, X, d, i, j);
}

/* ---------------------------------------------------------------------- */
/* One draw from w / sum(w):  j* = min{ j : C_j > U * W }.                  */
int64_t orc_sample(const double* w, int64_t N, double W, double U)
{
    double target = U * W;
    double c = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        c += w[j];
        if (w[j] > 0.0 && c > target) return j;
    }
    for (int64_t j = N - 1; j >= 0; --j)
        if (w[j] > 0.0) return j;
    return -1;
}

double orc_weight_total(const double* w, int64_t N)
{
    double W = 0.0;
    for (int64_t j = 0; j < N; ++j) W += w[j];
    return W;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (RejectionSampleSubmatrix) on the b x b psd matrix H
 * (row-major, overwritten).  u[i] is the proposal weight of proposal i,
 * uacc[i] its acceptance uniform.  At most max_accept pivots are accepted.
 * Outputs: acc[0..n) local indices of accepted proposals in order; Lc, an
 * n x n lower-triangular matrix (row-major, leading dimension b) with
 * H_in(acc,acc) = Lc Lc^*.                                                */
int orc_reject_chol(double* H, int32_t b, const double* u, const double* uacc,
                    int32_t max_accept, int32_t* acc, double* Lc, int32_t* n_out)
{
    if (b < 1 || !H || !u || !uacc || !acc || !Lc || !n_out) return ORC_EINVAL;
    double* L = (double*)calloc((size_t)b * b, sizeof(double));
    if (!L) return ORC_ENOMEM;
    int32_t n = 0;
    for (int32_t i = 0; i < b; ++i) {
        if (n >= max_accept) break;
        double hii = H[(int64_t)i * b + i];
        if (u[i] * uacc[i] < hii) {
            acc[n++] = i;
            double piv = sqrt(hii);
            for (int32_t j = i; j < b; ++j) L[(int64_t)j * b + i] = H[(int64_t)j * b + i] / piv;
            for (int32_t j = i + 1; j < b; ++j)
                for (int32_t l = i + 1; l <= j; ++l) {
                    double upd = L[(int64_t)j * b + i] * L[(int64_t)l * b + i];
                    H[(int64_t)j * b + l] -= upd;
                    if (l != j) H[(int64_t)l * b + j] -= upd;
                }
        }
    }
    for (int32_t a = 0; a < n; ++a)
        for (int32_t c = 0; c < b; ++c)
            Lc[(int64_t)a * b + c] = (c < n) ? L[(int64_t)acc[a] * b + acc[c]] : 0.0;
    *n_out = n;
    free(L);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 6, simple RPCholesky.  F is N x k, row-major, ld = k, zeroed by
 * the caller or here.  S receives the pivots.  d receives the final
 * (clamped) residual diagonal.  Returns the rank reached in *rank.        */
static int rpc_plain_impl(const orc_matrix* M, int64_t k, uint64_t seed, uint32_t inst,
                          double* F, int64_t* S, double* d, int64_t* rank_out)
{
    const int64_t N = M->N;
    if (k < 0 || k > N) return ORC_EINVAL;
    memset(F, 0, sizeof(double) * (size_t)N * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < N; ++j) d[j] = orc_entry(M, j, j);
    const double dfloor = orc_floor(d, N);
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    if (!g) return ORC_ENOMEM;
    int64_t rank = 0;
    for (int64_t step = 0; step < 4 * k + 64 && rank < k; ++step) {
        double W = orc_weight_total(d, N);
        if (!(W > 0.0)) break;
        double U;
        orc_uniform_pair(seed, 0u, (uint32_t)step, inst, &U, NULL);
        int64_t s = orc_sample(d, N, W, U);
        if (s < 0) break;
        const int64_t i = rank;
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double acc = orc_entry(M, r, s);
            for (int64_t m = 0; m < i; ++m) acc -= F[r * k + m] * F[s * k + m];
            g[r] = acc;
        }
        double gs = g[s];
        if (!(gs > 0.0)) {
            d[s] = 0.0;
            continue;
        }
        double piv = sqrt(gs);
        S[i] = s;
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double f = g[r] / piv;
            F[r * k + i] = f;
            double v = d[r] - f * f;
            d[r] = v > dfloor ? v : 0.0;
        }
        rank = i + 1;
    }
    free(g);
    *rank_out = rank;
    return ORC_OK;
}

/* Algorithm 2, accelerated RPCholesky with Algorithm 1 inside.
 * k: target rank (stop exactly there); T: block size b; max_rounds: stop
 * after this many rounds (<= 0: no limit besides k).  F: N x k row-major,
 * ld = k.  Per-round sizes are written to round_sizes (if not NULL, length
 * >= number of rounds).  accept_rule 0: u_i = d[s'_i] (proposal weight);
 * 1: u_i = h_ii at entry of Algorithm 1 (the literal line of Algorithm 1).
 * dpre (if not NULL) receives the residual diagonal of the last round
 * before clamping.                                                        */
static int rpc_accel_impl(const orc_matrix* M, int64_t k, int32_t T, int64_t max_rounds,
                          uint64_t seed, uint32_t inst, int accept_rule, double* F, int64_t* S,
                          double* d, double* dpre, int64_t* rank_out, int64_t* rounds_out,
                          int32_t* round_sizes, int64_t round_sizes_cap)
{
    const int64_t N = M->N;
    if (k < 0 || k > N || T < 1) return ORC_EINVAL;
    memset(F, 0, sizeof(double) * (size_t)N * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < N; ++j) {
        d[j] = orc_entry(M, j, j);
        if (dpre) dpre[j] = d[j];
    }
    const double dfloor = orc_floor(d, N);
    int64_t* prop = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    double* u = (double*)malloc(sizeof(double) * (size_t)T);
    double* ua = (double*)malloc(sizeof(double) * (size_t)T);
    double* H = (double*)malloc(sizeof(double) * (size_t)T * T);
    double* L = (double*)malloc(sizeof(double) * (size_t)T * T);
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)T);
    int64_t* Si = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    if (!prop || !u || !ua || !H || !L || !acc || !Si) {
        free(prop); free(u); free(ua); free(H); free(L); free(acc); free(Si);
        return ORC_ENOMEM;
    }
    int64_t rank = 0, round = 0;
    while (rank < k && (max_rounds <= 0 || round < max_rounds)) {
        /* Step 1: propose T iid pivots from u = d. */
        double W = orc_weight_total(d, N);
        if (!(W > 0.0)) break;
        for (int32_t j = 0; j < T; ++j) {
            double Up, Ua;
            orc_uniform_pair(seed, (uint32_t)j, (uint32_t)round, inst, &Up, &Ua);
            prop[j] = orc_sample(d, N, W, Up);
            u[j] = d[prop[j]];
            ua[j] = Ua;
        }
        /* Step 2: H = A(S',S') - F(S',:) F(S',:)^*, then Algorithm 1. */
        for (int32_t a = 0; a < T; ++a)
            for (int32_t b = 0; b < T; ++b) {
                double h = orc_entry(M, prop[a], prop[b]);
                for (int64_t m = 0; m < rank; ++m) h -= F[prop[a] * k + m] * F[prop[b] * k + m];
                H[(int64_t)a * T + b] = h;
            }
        if (accept_rule == 1)
            for (int32_t a = 0; a < T; ++a) u[a] = H[(int64_t)a * T + a];
        int32_t n = 0;
        int rc = orc_reject_chol(H, T, u, ua, (int32_t)(k - rank), acc, L, &n);
        if (rc != ORC_OK) {
            free(prop); free(u); free(ua); free(H); free(L); free(acc); free(Si);
            return rc;
        }
        if (round_sizes && round < round_sizes_cap) round_sizes[round] = n;
        for (int32_t a = 0; a < n; ++a) {
            Si[a] = prop[acc[a]];
            S[rank + a] = Si[a];
        }
        /* Step 3: G = (A(:,S_i) - F F(S_i,:)^*) L^{-*}; F <- [F G];
         *         u <- max(u - rowsumsq(G), 0).                           */
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double Grow[1024];
            double* G = Grow;
            double* Gheap = NULL;
            if (n > 1024) {
                Gheap = (double*)malloc(sizeof(double) * (size_t)n);
                G = Gheap;
            }
            for (int32_t j = 0; j < n; ++j) {
                double rr = orc_entry(M, r, Si[j]);
                for (int64_t m = 0; m < rank; ++m) rr -= F[r * k + m] * F[Si[j] * k + m];
                G[j] = rr;
            }
            for (int32_t j = 0; j < n; ++j) {
                double v = G[j];
                for (int32_t l = 0; l < j; ++l) v -= G[l] * L[(int64_t)j * T + l];
                G[j] = v / L[(int64_t)j * T + j];
            }
            double rsq = 0.0;
            for (int32_t j = 0; j < n; ++j) {
                F[r * k + rank + j] = G[j];
                rsq += G[j] * G[j];
            }
            double v = d[r] - rsq;
            if (dpre) dpre[r] = v;
            d[r] = v > dfloor ? v : 0.0;
            free(Gheap);
        }
        rank += n;
        round += 1;
    }
    free(prop); free(u); free(ua); free(H); free(L); free(acc); free(Si);
    *rank_out = rank;
    if (rounds_out) *rounds_out = round;
    return ORC_OK;
}

/* Algorithm 7 (appendix), block RPCholesky: per round, b iid draws from
 * d / sum(d), Unique, G = A(:,S') - F F(S',:)^*, R = Chol(G(S',:)),
 * F(:, new) = G R^{-1}, d <- max(d - rowsumsq, 0).  Readings:
 *   - the draws use the same Philox blocks as Algorithm 2 (slot j, round r,
 *     proposal words), so that b = 1 meets Algorithm 6 step for step;
 *   - Unique keeps the first draw of each index, in draw order;
 *   - Chol is the semidefinite Cholesky in that order: a pivot whose Schur
 *     residual is not positive gets a zero column, and the algorithm's last
 *     line (remove zero columns) drops it; at most k - rank pivots are kept.
 * Arguments as for rpc_accel_impl.                                        */
static int rpc_block_impl(const orc_matrix* M, int64_t k, int32_t b, int64_t max_rounds,
                          uint64_t seed, uint32_t inst, double* F, int64_t* S, double* d,
                          int64_t* rank_out, int64_t* rounds_out, int32_t* round_sizes,
                          int64_t round_sizes_cap)
{
    const int64_t N = M->N;
    if (k < 0 || k > N || b < 1) return ORC_EINVAL;
    memset(F, 0, sizeof(double) * (size_t)N * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < N; ++j) d[j] = orc_entry(M, j, j);
    const double dfloor = orc_floor(d, N);
    int64_t* Su = (int64_t*)malloc(sizeof(int64_t) * (size_t)b);   /* S' after Unique */
    double* Gs = (double*)malloc(sizeof(double) * (size_t)b * b);  /* G(S',:), then R^* */
    int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)b);
    if (!Su || !Gs || !keep) {
        free(Su); free(Gs); free(keep);
        return ORC_ENOMEM;
    }
    int64_t rank = 0, round = 0;
    while (rank < k && (max_rounds <= 0 || round < max_rounds)) {
        double W = orc_weight_total(d, N);
        if (!(W > 0.0)) break;
        /* b iid draws, then Unique */
        int32_t m = 0;
        for (int32_t j = 0; j < b; ++j) {
            double Up;
            orc_uniform_pair(seed, (uint32_t)j, (uint32_t)round, inst, &Up, NULL);
            int64_t s = orc_sample(d, N, W, Up);
            int seen = 0;
            for (int32_t a = 0; a < m; ++a) seen |= Su[a] == s;
            if (!seen) Su[m++] = s;
        }
        /* G(S',:) = A(S',S') - F(S',:) F(S',:)^* */
        for (int32_t a = 0; a < m; ++a)
            for (int32_t c = 0; c < m; ++c) {
                double g = orc_entry(M, Su[a], Su[c]);
                for (int64_t l = 0; l < rank; ++l) g -= F[Su[a] * k + l] * F[Su[c] * k + l];
                Gs[(int64_t)a * m + c] = g;
            }
        /* semidefinite Cholesky, in place: the lower triangle becomes R^*
         * on the kept columns; a dropped pivot leaves its column unused   */
        int32_t n = 0;
        for (int32_t i = 0; i < m; ++i) {
            double gii = Gs[(int64_t)i * m + i];
            if (n >= k - rank || !(gii > dfloor)) continue;  /* no pivot on rounding noise */
            keep[n++] = i;
            double piv = sqrt(gii);
            for (int32_t j = i; j < m; ++j) Gs[(int64_t)j * m + i] /= piv;
            for (int32_t j = i + 1; j < m; ++j)
                for (int32_t l = i + 1; l <= j; ++l)
                    Gs[(int64_t)j * m + l] -= Gs[(int64_t)j * m + i] * Gs[(int64_t)l * m + i];
        }
        if (round_sizes && round < round_sizes_cap) round_sizes[round] = n;
        for (int32_t a = 0; a < n; ++a) S[rank + a] = Su[keep[a]];
        /* F(r, new) = G(r, kept) R^{-1}: forward substitution with R^* */
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double Grow[1024];
            double* G = Grow;
            double* Gheap = NULL;
            if (n > 1024) {
                Gheap = (double*)malloc(sizeof(double) * (size_t)n);
                G = Gheap;
            }
            double rsq = 0.0;
            for (int32_t a = 0; a < n; ++a) {
                const int64_t s = Su[keep[a]];
                double v = orc_entry(M, r, s);
                for (int64_t l = 0; l < rank; ++l) v -= F[r * k + l] * F[s * k + l];
                for (int32_t c = 0; c < a; ++c)
                    v -= G[c] * Gs[(int64_t)keep[a] * m + keep[c]];
                G[a] = v / Gs[(int64_t)keep[a] * m + keep[a]];
            }
            for (int32_t a = 0; a < n; ++a) {
                F[r * k + rank + a] = G[a];
                rsq += G[a] * G[a];
            }
            double v = d[r] - rsq;
            d[r] = v > dfloor ? v : 0.0;
            free(Gheap);
        }
        rank += n;
        round += 1;
    }
    free(Su); free(Gs); free(keep);
    *rank_out = rank;
    if (rounds_out) *rounds_out = round;
    return ORC_OK;
}

/* Algorithm 3, the low-memory form of Algorithm 2: no N x k factor is kept,
 * only the pivots S and the Cholesky factor L of A(S,S) (k x k, row-major,
 * leading dimension k).  Per round:
 *   Step 1: the same T draws as Algorithm 2 (same Philox blocks);
 *   Step 2: H = A(S',S') - Y^* Y with Y = L^{-1} A(S,S') (forward
 *           substitution), then Algorithm 1 on H;
 *   Step 3: for every row r (the listing's row chunks cover all N rows):
 *           g = A(r,S_i) - A(r,S_old) M with M = L^{-*} Y(:,acc) formed once
 *           per round (back substitution), G(r,:) = g L_i^{-*} (forward
 *           substitution with L_i), u(r) -= |G(r,:)|^2;
 *           L <- [L 0; Y(:,acc)^* L_i]; u <- max(u, 0).
 * d receives u; Lout the k x k factor (zero beyond rank).                 */
static int rpc_lowmem_impl(const orc_matrix* M, int64_t k, int32_t T, int64_t max_rounds,
                           uint64_t seed, uint32_t inst, double* Lout, int64_t* S, double* d,
                           int64_t* rank_out, int64_t* rounds_out)
{
    const int64_t N = M->N;
    if (k < 0 || k > N || T < 1) return ORC_EINVAL;
    const int64_t kk = k > 0 ? k : 1;
    memset(Lout, 0, sizeof(double) * (size_t)kk * (size_t)kk);
    for (int64_t j = 0; j < N; ++j) d[j] = orc_entry(M, j, j);
    const double dfloor = orc_floor(d, N);
    int64_t* prop = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    double* u = (double*)malloc(sizeof(double) * (size_t)T);
    double* ua = (double*)malloc(sizeof(double) * (size_t)T);
    double* H = (double*)malloc(sizeof(double) * (size_t)T * T);
    double* Li = (double*)malloc(sizeof(double) * (size_t)T * T);
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)T);
    double* Y = (double*)malloc(sizeof(double) * (size_t)T * kk);   /* Y(:,j) at Y + j*k */
    double* Mm = (double*)malloc(sizeof(double) * (size_t)T * kk);  /* M(:,a) at Mm + a*k */
    if (!prop || !u || !ua || !H || !Li || !acc || !Y || !Mm) {
        free(prop); free(u); free(ua); free(H); free(Li); free(acc); free(Y); free(Mm);
        return ORC_ENOMEM;
    }
    int64_t rank = 0, round = 0;
    while (rank < k && (max_rounds <= 0 || round < max_rounds)) {
        double W = orc_weight_total(d, N);
        if (!(W > 0.0)) break;
        for (int32_t j = 0; j < T; ++j) {
            double Up, Ua;
            orc_uniform_pair(seed, (uint32_t)j, (uint32_t)round, inst, &Up, &Ua);
            prop[j] = orc_sample(d, N, W, Up);
            u[j] = d[prop[j]];
            ua[j] = Ua;
        }
        /* Y(:,j) = L^{-1} A(S, s'_j) */
        for (int32_t j = 0; j < T; ++j) {
            double* y = Y + (int64_t)j * kk;
            for (int64_t m = 0; m < rank; ++m) {
                double v = orc_entry(M, S[m], prop[j]);
                for (int64_t l = 0; l < m; ++l) v -= Lout[m * kk + l] * y[l];
                y[m] = v / Lout[m * kk + m];
            }
        }
        for (int32_t a = 0; a < T; ++a)
            for (int32_t c = 0; c < T; ++c) {
                double h = orc_entry(M, prop[a], prop[c]);
                for (int64_t m = 0; m < rank; ++m) h -= Y[(int64_t)a * kk + m] * Y[(int64_t)c * kk + m];
                H[(int64_t)a * T + c] = h;
            }
        int32_t n = 0;
        int rc = orc_reject_chol(H, T, u, ua, (int32_t)(k - rank), acc, Li, &n);
        if (rc != ORC_OK) {
            free(prop); free(u); free(ua); free(H); free(Li); free(acc); free(Y); free(Mm);
            return rc;
        }
        /* M(:,a) = L^{-*} Y(:, acc_a) */
        for (int32_t a = 0; a < n; ++a) {
            const double* y = Y + (int64_t)acc[a] * kk;
            double* z = Mm + (int64_t)a * kk;
            for (int64_t m = rank - 1; m >= 0; --m) {
                double v = y[m];
                for (int64_t l = m + 1; l < rank; ++l) v -= Lout[l * kk + m] * z[l];
                z[m] = v / Lout[m * kk + m];
            }
        }
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double gbuf[1024];
            double* g = gbuf;
            double* gheap = NULL;
            if (n > 1024) {
                gheap = (double*)malloc(sizeof(double) * (size_t)n);
                g = gheap;
            }
            for (int32_t a = 0; a < n; ++a) {
                double v = orc_entry(M, r, prop[acc[a]]);
                for (int64_t m = 0; m < rank; ++m)
                    v -= orc_entry(M, r, S[m]) * Mm[(int64_t)a * kk + m];
                g[a] = v;
            }
            double rsq = 0.0;
            for (int32_t a = 0; a < n; ++a) {
                double v = g[a];
                for (int32_t c = 0; c < a; ++c) v -= g[c] * Li[(int64_t)a * T + c];
                g[a] = v / Li[(int64_t)a * T + a];
                rsq += g[a] * g[a];
            }
            double v = d[r] - rsq;
            d[r] = v > dfloor ? v : 0.0;
            free(gheap);
        }
        /* L <- [L 0; Y(:,acc)^* L_i] */
        for (int32_t a = 0; a < n; ++a) {
            for (int64_t m = 0; m < rank; ++m)
                Lout[(rank + a) * kk + m] = Y[(int64_t)acc[a] * kk + m];
            for (int32_t c = 0; c <= a; ++c)
                Lout[(rank + a) * kk + rank + c] = Li[(int64_t)a * T + c];
            S[rank + a] = prop[acc[a]];
        }
        rank += n;
        round += 1;
    }
    free(prop); free(u); free(ua); free(H); free(Li); free(acc); free(Y); free(Mm);
    *rank_out = rank;
    if (rounds_out) *rounds_out = round;
    return ORC_OK;
}

/* Algorithm 5, accelerated randomly pivoted QR of a dense B (M x N,
 * column-major: column j at B + j*M).  u starts at the squared column norms.
 * Per round: the T draws of Algorithm 2 (same Philox blocks; u_i = u[s'_i]),
 * C = B(:,S') - Q F(S',:)^*, Algorithm 1 on C^* C (its L discarded),
 * Q_perp = C(:, acc) (= B(:,S_i) - Q F(S_i,:)^*), one more Gram-Schmidt pass
 * Q_perp -= Q (Q^* Q_perp), Orth = the Q factor of the thin QR with positive
 * diagonal, formed by classical Gram-Schmidt applied twice column by column;
 * Q <- [Q Q_perp], G = B^* Q_perp, F <- [F G], u <- max(u - rowsumsq(G), 0).
 * Q: M x k column-major (ld M); F: N x k row-major (ld k).                 */
static int rpqr_accel_impl(const double* B, int64_t M, int64_t N, int64_t k, int32_t T,
                           int64_t max_rounds, uint64_t seed, uint32_t inst, double* Q,
                           double* F, int64_t* S, double* u, int64_t* rank_out,
                           int64_t* rounds_out)
{
    if (k < 0 || k > N || k > M || T < 1 || M < 1) return ORC_EINVAL;
    const int64_t kk = k > 0 ? k : 1;
    memset(Q, 0, sizeof(double) * (size_t)M * (size_t)kk);
    memset(F, 0, sizeof(double) * (size_t)N * (size_t)kk);
    for (int64_t j = 0; j < N; ++j) {
        double t = 0.0;
        for (int64_t i = 0; i < M; ++i) t += B[j * M + i] * B[j * M + i];
        u[j] = t;
    }
    int64_t* prop = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    double* up = (double*)malloc(sizeof(double) * (size_t)T);
    double* ua = (double*)malloc(sizeof(double) * (size_t)T);
    double* C = (double*)malloc(sizeof(double) * (size_t)M * T);
    double* H = (double*)malloc(sizeof(double) * (size_t)T * T);
    double* L = (double*)malloc(sizeof(double) * (size_t)T * T);
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)T);
    double* w = (double*)malloc(sizeof(double) * (size_t)(kk + T));
    if (!prop || !up || !ua || !C || !H || !L || !acc || !w) {
        free(prop); free(up); free(ua); free(C); free(H); free(L); free(acc); free(w);
        return ORC_ENOMEM;
    }
    int64_t rank = 0, round = 0;
    while (rank < k && (max_rounds <= 0 || round < max_rounds)) {
        double W = orc_weight_total(u, N);
        if (!(W > 0.0)) break;
        for (int32_t j = 0; j < T; ++j) {
            double Up, Ua;
            orc_uniform_pair(seed, (uint32_t)j, (uint32_t)round, inst, &Up, &Ua);
            prop[j] = orc_sample(u, N, W, Up);
            up[j] = u[prop[j]];
            ua[j] = Ua;
        }
        /* C = B(:,S') - Q F(S',:)^* */
        for (int32_t a = 0; a < T; ++a)
            for (int64_t i = 0; i < M; ++i) {
                double v = B[prop[a] * M + i];
                for (int64_t m = 0; m < rank; ++m) v -= Q[m * M + i] * F[prop[a] * kk + m];
                C[(int64_t)a * M + i] = v;
            }
        for (int32_t a = 0; a < T; ++a)
            for (int32_t c = 0; c < T; ++c) {
                double h = 0.0;
                for (int64_t i = 0; i < M; ++i) h += C[(int64_t)a * M + i] * C[(int64_t)c * M + i];
                H[(int64_t)a * T + c] = h;
            }
        int32_t n = 0;
        int rc = orc_reject_chol(H, T, up, ua, (int32_t)(k - rank), acc, L, &n);
        if (rc != ORC_OK) {
            free(prop); free(up); free(ua); free(C); free(H); free(L); free(acc); free(w);
            return rc;
        }
        /* Q_perp = C(:,acc) into Q(:, rank:rank+n), re-orthogonalised against Q */
        for (int32_t a = 0; a < n; ++a) {
            double* q = Q + (rank + a) * M;
            memcpy(q, C + (int64_t)acc[a] * M, sizeof(double) * (size_t)M);
            S[rank + a] = prop[acc[a]];
        }
        for (int32_t a = 0; a < n; ++a) {
            double* q = Q + (rank + a) * M;
            for (int64_t m = 0; m < rank; ++m) {
                double t = 0.0;
                for (int64_t i = 0; i < M; ++i) t += Q[m * M + i] * q[i];
                w[m] = t;
            }
            for (int64_t i = 0; i < M; ++i) {
                double v = q[i];
                for (int64_t m = 0; m < rank; ++m) v -= Q[m * M + i] * w[m];
                q[i] = v;
            }
        }
        /* Orth: column a against columns rank..rank+a-1, twice, then normalised */
        for (int32_t a = 0; a < n; ++a) {
            double* q = Q + (rank + a) * M;
            for (int pass = 0; pass < 2; ++pass) {
                for (int32_t c = 0; c < a; ++c) {
                    const double* qc = Q + (rank + c) * M;
                    double t = 0.0;
                    for (int64_t i = 0; i < M; ++i) t += qc[i] * q[i];
                    w[c] = t;
                }
                for (int64_t i = 0; i < M; ++i) {
                    double v = q[i];
                    for (int32_t c = 0; c < a; ++c) v -= Q[(rank + c) * M + i] * w[c];
                    q[i] = v;
                }
            }
            double nrm = 0.0;
            for (int64_t i = 0; i < M; ++i) nrm += q[i] * q[i];
            nrm = sqrt(nrm);
            for (int64_t i = 0; i < M; ++i) q[i] /= nrm;
        }
        /* G = B^* Q_perp; F <- [F G]; u update */
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            double rsq = 0.0;
            for (int32_t a = 0; a < n; ++a) {
                const double* q = Q + (rank + a) * M;
                double g = 0.0;
                for (int64_t i = 0; i < M; ++i) g += B[j * M + i] * q[i];
                F[j * kk + rank + a] = g;
                rsq += g * g;
            }
            double v = u[j] - rsq;
            u[j] = v > 0.0 ? v : 0.0;
        }
        rank += n;
        round += 1;
    }
    free(prop); free(up); free(ua); free(C); free(H); free(L); free(acc); free(w);
    *rank_out = rank;
    if (rounds_out) *rounds_out = round;
    return ORC_OK;
}

int orc_rpqr_accel(const double* B, int64_t M, int64_t N, int64_t k, int32_t T,
                   int64_t max_rounds, uint64_t seed, uint32_t inst, double* Q, double* F,
                   int64_t* S, double* u, int64_t* rank, int64_t* rounds)
{
    if (!B || !Q || !F || !S || !u || !rank) return ORC_EINVAL;
    return rpqr_accel_impl(B, M, N, k, T, max_rounds, seed, inst, Q, F, S, u, rank, rounds);
}

/* Cholesky with the given pivot order (the deterministic recursion of
 * Algorithm 6 with s_i fixed): F is N x k row-major (ld = k); d receives
 * diag(A - F F^*).  A pivot whose residual is <= 0 adds a zero column.
 * Returns tr(A - F F^*) in *trace_err.                                    */
static int fixed_pivot_impl(const orc_matrix* M, const int64_t* S, int64_t k, double* F,
                            double* d, double* trace_err)
{
    const int64_t N = M->N;
    memset(F, 0, sizeof(double) * (size_t)N * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < N; ++j) d[j] = orc_entry(M, j, j);
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    if (!g) return ORC_ENOMEM;
    for (int64_t i = 0; i < k; ++i) {
        int64_t s = S[i];
        if (s < 0 || s >= N) {
            free(g);
            return ORC_EINVAL;
        }
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t r = 0; r < N; ++r) {
            double acc = orc_entry(M, r, s);
            for (int64_t m = 0; m < i; ++m) acc -= F[r * k + m] * F[s * k + m];
            g[r] = acc;
        }
        double gs = g[s];
        if (!(gs > 0.0)) continue;
        double piv = sqrt(gs);
        for (int64_t r = 0; r < N; ++r) {
            double f = g[r] / piv;
            F[r * k + i] = f;
            d[r] -= f * f;
        }
    }
    double t = 0.0;
    for (int64_t j = 0; j < N; ++j) t += d[j];
    *trace_err = t;
    free(g);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Exported entry points.  X: N x d float row-major (points) or NULL;
 * A: N x N double row-major (explicit psd matrix) or NULL; exactly one of
 * the two is given.                                                       */
static int make_matrix(orc_matrix* M, const float* X, int d, int kind, double sigma,
                       const double* A, int64_t N)
{
    if (N < 1) return ORC_EINVAL;
    if ((X == NULL) == (A == NULL)) return ORC_EINVAL;
    if (X && (d < 1 || !(sigma > 0.0) || kind < 0 || kind > 4)) return ORC_EINVAL;
    M->X = X;
    M->d = d;
    M->kind = kind;
    M->sigma = sigma;
    M->A = A;
    M->N = N;
    return ORC_OK;
}

int orc_rpc_plain(const float* X, int d, int kind, double sigma, const double* A, int64_t N,
                  int64_t k, uint64_t seed, uint32_t inst, double* F, int64_t* S, double* dres,
                  int64_t* rank)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    return rpc_plain_impl(&M, k, seed, inst, F, S, dres, rank);
}

int orc_rpc_accel(const float* X, int d, int kind, double sigma, const double* A, int64_t N,
                  int64_t k, int32_t T, int64_t max_rounds, uint64_t seed, uint32_t inst,
                  int accept_rule, double* F, int64_t* S, double* dres, double* dpre,
                  int64_t* rank, int64_t* rounds, int32_t* round_sizes, int64_t round_sizes_cap)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    return rpc_accel_impl(&M, k, T, max_rounds, seed, inst, accept_rule, F, S, dres, dpre, rank,
                          rounds, round_sizes, round_sizes_cap);
}

int orc_rpc_block(const float* X, int d, int kind, double sigma, const double* A, int64_t N,
                  int64_t k, int32_t b, int64_t max_rounds, uint64_t seed, uint32_t inst,
                  double* F, int64_t* S, double* dres, int64_t* rank, int64_t* rounds,
                  int32_t* round_sizes, int64_t round_sizes_cap)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    return rpc_block_impl(&M, k, b, max_rounds, seed, inst, F, S, dres, rank, rounds,
                          round_sizes, round_sizes_cap);
}

int orc_rpc_lowmem(const float* X, int d, int kind, double sigma, const double* A, int64_t N,
                   int64_t k, int32_t T, int64_t max_rounds, uint64_t seed, uint32_t inst,
                   double* L, int64_t* S, double* dres, int64_t* rank, int64_t* rounds)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    return rpc_lowmem_impl(&M, k, T, max_rounds, seed, inst, L, S, dres, rank, rounds);
}

int orc_fixed_pivot_factor(const float* X, int d, int kind, double sigma, const double* A,
                           int64_t N, const int64_t* S, int64_t k, double* F, double* dres,
                           double* trace_err)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    return fixed_pivot_impl(&M, S, k, F, dres, trace_err);
}

/* Many independent runs on one matrix (instances inst0 .. inst0+n-1), for
 * the distribution tests; only the first k pivots of each are kept.
 * algo 0: simple RPCholesky; algo 1: accelerated with block T.            */
int orc_pivots_many(const float* X, int d, int kind, double sigma, const double* A, int64_t N,
                    int algo, int64_t k, int32_t T, uint64_t seed, uint32_t inst0, int64_t n,
                    int64_t* S_out, int64_t* rank_out)
{
    orc_matrix M;
    int rc = make_matrix(&M, X, d, kind, sigma, A, N);
    if (rc) return rc;
    double* F = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(k > 0 ? k : 1));
    double* dd = (double*)malloc(sizeof(double) * (size_t)N);
    if (!F || !dd) {
        free(F);
        free(dd);
        return ORC_ENOMEM;
    }
    for (int64_t t = 0; t < n; ++t) {
        int64_t rank = 0;
        uint32_t inst = inst0 + (uint32_t)t;
        if (algo == 0)
            rc = rpc_plain_impl(&M, k, seed, inst, F, S_out + t * k, dd, &rank);
        else
            rc = rpc_accel_impl(&M, k, T, 0, seed, inst, 0, F, S_out + t * k, dd, NULL, &rank,
                                NULL, NULL, 0);
        if (rc) break;
        rank_out[t] = rank;
    }
    free(F);
    free(dd);
    return rc;
}

/* Residual trace after t rounds of accelerated RPCholesky for many runs
 * (Lemma "central error bound" check).                                    */
int orc_accel_trace_many(const double* A, int64_t N, int32_t T, int64_t rounds, uint64_t seed,
                         uint32_t inst0, int64_t n, double* trace_out)
{
    orc_matrix M;
    int rc = make_matrix(&M, NULL, 0, 0, 1.0, A, N);
    if (rc) return rc;
    double* F = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
    double* dd = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    if (!F || !dd || !S) {
        free(F); free(dd); free(S);
        return ORC_ENOMEM;
    }
    for (int64_t t = 0; t < n; ++t) {
        int64_t rank = 0, nr = 0;
        rc = rpc_accel_impl(&M, N, T, rounds, seed, inst0 + (uint32_t)t, 0, F, S, dd, NULL, &rank,
                            &nr, NULL, 0);
        if (rc) break;
        /* exact residual trace from the factor: tr(A) - ||F||_F^2 */
        double tr = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double v = A[j * N + j];
            for (int64_t m = 0; m < rank; ++m) v -= F[j * N + m] * F[j * N + m];
            tr += v;
        }
        trace_out[t] = tr;
    }
    free(F); free(dd); free(S);
    return rc;
}
