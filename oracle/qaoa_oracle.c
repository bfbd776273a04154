/*
 * CPU oracle for the AA-QAOA hot path -- test infrastructure only.
 *
 * This file is the plain, slow, FP64 (C99 double complex) statement of what
 * the CUDA path computes. It exists so that tests, the package's smoke check
 * and the benchmark's CPU baseline have an independent answer to compare
 * against; no product code links or calls it. It shares no code, tables or
 * headers with the CUDA library.
 *
 * Conventions (the paper leaves them implicit):
 *   - qubit i is bit i of the basis-state index x (little-endian);
 *   - the ansatz is Eq. (1) read literally: layer l applies exp(-i gamma_l H_C)
 *     then exp(-i beta_l H_M), and layer 1 acts first on |+>^n, as Eq. (A2)
 *     writes the product out;
 *   - H_C = 1/2 sum_{(i,j) in E} (1 - Z_i Z_j) (Eq. for H_P with unit weights),
 *     whose diagonal is the integer cut count C(x);
 *   - H_M = sum_i X_i, so exp(-i beta H_M) = prod_i RX_i(2 beta) with
 *     RX(2 beta) = [[cos b, -i sin b], [-i sin b, cos b]];
 *   - an observable is a weighted list of edges (u, v, w) standing for
 *     1/2 sum w (1 - Z_u Z_v). With every edge at weight 1 it is H_C; with the
 *     orbit representatives at weight |S~_m| it is H_red (Sec. 5, "Reducing the Hamiltonian").
 *
 * Nothing is blocked, fused or reordered: each function is the textbook loop
 * over basis states. The "#pragma omp" lines mark loops whose iterations are
 * independent (or a plain sum); the pinned oracle is compiled without OpenMP,
 * which ignores them. A separate -fopenmp build of this same file serves only
 * to time the oracle on all host cores (its sums then run in another order).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Cut count C(x) = sum over edges of [x_u != x_v]: the diagonal of H_C,
 * edge by edge (Eq. for H_P, unit weights). */
int64_t oracle_cut_value(int m, const int32_t *edges, uint64_t x)
{
    int64_t c = 0;
    for (int e = 0; e < m; e++) {
        uint64_t bu = (x >> edges[2 * e]) & 1u;
        uint64_t bv = (x >> edges[2 * e + 1]) & 1u;
        c += (bu != bv);
    }
    return c;
}

/* Diagonal of a weighted observable 1/2 sum_k w_k (1 - Z_{u_k} Z_{v_k}) at x:
 * sum_k w_k [x_{u_k} != x_{v_k}]. With the orbit representatives and orbit
 * sizes this is the diagonal of H_red (Sec. 5, equation for H_red). */
double oracle_observable_value(int k, const int32_t *obs_edges, const double *w, uint64_t x)
{
    double s = 0.0;
    for (int e = 0; e < k; e++) {
        uint64_t bu = (x >> obs_edges[2 * e]) & 1u;
        uint64_t bv = (x >> obs_edges[2 * e + 1]) & 1u;
        if (bu != bv)
            s += w[e];
    }
    return s;
}

/* |+>^n: every amplitude 2^{-n/2} (initial state of Eq. (1)). */
void oracle_plus_state(int n, cplx *psi)
{
    uint64_t N = 1ull << n;
    double a = 1.0 / sqrt((double)N);
#pragma omp parallel for
    for (uint64_t x = 0; x < N; x++)
        psi[x] = a;
}

/* psi <- exp(-i gamma H_C) psi: a phase exp(-i gamma C(x)) on each amplitude. */
void oracle_apply_cost(int n, int m, const int32_t *edges, double gamma, cplx *psi)
{
    uint64_t N = 1ull << n;
#pragma omp parallel for
    for (uint64_t x = 0; x < N; x++) {
        double c = (double)oracle_cut_value(m, edges, x);
        psi[x] *= cexp(-I * gamma * c);
    }
}

/* psi <- RX_q(2 beta) psi = exp(-i beta X_q) psi on one qubit q. */
void oracle_apply_rx(int n, int q, double beta, cplx *psi)
{
    uint64_t N = 1ull << n, bit = 1ull << q;
    double c = cos(beta), s = sin(beta);
#pragma omp parallel for
    for (uint64_t x = 0; x < N; x++) {
        if (x & bit)
            continue;
        cplx a = psi[x], b = psi[x | bit];
        psi[x] = c * a - I * s * b;
        psi[x | bit] = -I * s * a + c * b;
    }
}

/* psi <- exp(-i beta H_M) psi with H_M = sum_i X_i (mixer of Eq. (1)). */
void oracle_apply_mixer(int n, double beta, cplx *psi)
{
    for (int q = 0; q < n; q++)
        oracle_apply_rx(n, q, beta, psi);
}

/* The p-layer QAOA state of Eq. (1): layer 1 first (Eq. (A2)). */
void oracle_qaoa_state(int n, int m, const int32_t *edges, int p,
                       const double *gamma, const double *beta, cplx *psi)
{
    oracle_plus_state(n, psi);
    for (int l = 0; l < p; l++) {
        oracle_apply_cost(n, m, edges, gamma[l], psi);
        oracle_apply_mixer(n, beta[l], psi);
    }
}

/* <psi| O |psi> for the diagonal observable O(x) of oracle_observable_value:
 * sum_x |psi_x|^2 O(x) (cost function F_p of Eq. (2)). */
double oracle_expect_diag(int n, const cplx *psi, int k, const int32_t *obs_edges, const double *w)
{
    uint64_t N = 1ull << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (uint64_t x = 0; x < N; x++) {
        double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        s += pr * oracle_observable_value(k, obs_edges, w, x);
    }
    return s;
}

/* <psi| Z_u Z_v |psi> = sum_x |psi_x|^2 (-1)^{x_u + x_v}: one term of the
 * estimator aggregation, one pass over the amplitudes (Eq. (agg)). */
double oracle_zz(int n, const cplx *psi, int u, int v)
{
    uint64_t N = 1ull << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (uint64_t x = 0; x < N; x++) {
        double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        int sign = (((x >> u) ^ (x >> v)) & 1u) ? -1 : 1;
        s += sign * pr;
    }
    return s;
}

/* Estimator aggregation term by term (Eq. (agg) and its reduced form):
 * sum_k w_k * 1/2 (1 - <Z_{u_k} Z_{v_k}>), one pass over psi per term. */
double oracle_expect_terms(int n, const cplx *psi, int k, const int32_t *obs_edges, const double *w)
{
    double s = 0.0;
    for (int e = 0; e < k; e++)
        s += w[e] * 0.5 * (1.0 - oracle_zz(n, psi, obs_edges[2 * e], obs_edges[2 * e + 1]));
    return s;
}

/* Energy and its gradient by the adjoint recursion.
 *
 * E = <psi|O|psi> with psi = U_p ... U_1 |+>, U_l = exp(-i b_l H_M) exp(-i g_l H_C).
 * With phi = psi and lambda = O psi, for l = p .. 1:
 *   dE/db_l = 2 Im <lambda| H_M |phi>;
 *   phi, lambda <- exp(+i b_l H_M) phi, lambda;
 *   dE/dg_l = 2 Im <lambda| H_C |phi>;
 *   phi, lambda <- exp(+i g_l H_C) phi, lambda.
 * (Derivative of the cost function F_p of Eq. (2).) phi and lam are caller
 * buffers of 2^n amplitudes. Returns E.
 */
double oracle_energy_grad(int n, int m, const int32_t *edges, int p,
                          const double *gamma, const double *beta,
                          int k, const int32_t *obs_edges, const double *w,
                          double *dgamma, double *dbeta, cplx *phi, cplx *lam)
{
    uint64_t N = 1ull << n;
    oracle_qaoa_state(n, m, edges, p, gamma, beta, phi);
    double energy = 0.0;
#pragma omp parallel for reduction(+ : energy)
    for (uint64_t x = 0; x < N; x++) {
        double o = oracle_observable_value(k, obs_edges, w, x);
        lam[x] = o * phi[x];
        energy += o * (creal(phi[x]) * creal(phi[x]) + cimag(phi[x]) * cimag(phi[x]));
    }
    for (int l = p - 1; l >= 0; l--) {
        /* <lambda| sum_i X_i |phi>; only its imaginary part is used */
        double acc_im = 0.0;
        for (int q = 0; q < n; q++) {
            uint64_t bit = 1ull << q;
#pragma omp parallel for reduction(+ : acc_im)
            for (uint64_t x = 0; x < N; x++)
                acc_im += cimag(conj(lam[x]) * phi[x ^ bit]);
        }
        dbeta[l] = 2.0 * acc_im;
        oracle_apply_mixer(n, -beta[l], phi);
        oracle_apply_mixer(n, -beta[l], lam);
        /* <lambda| H_C |phi>; only its imaginary part is used */
        acc_im = 0.0;
#pragma omp parallel for reduction(+ : acc_im)
        for (uint64_t x = 0; x < N; x++)
            acc_im += cimag(conj(lam[x]) * (double)oracle_cut_value(m, edges, x) * phi[x]);
        dgamma[l] = 2.0 * acc_im;
        oracle_apply_cost(n, m, edges, -gamma[l], phi);
        oracle_apply_cost(n, m, edges, -gamma[l], lam);
    }
    return energy;
}

/* Maximum cut C_max = max_x C(x) by exhaustion over all 2^n basis states, and
 * the smallest x attaining it: the denominator of the approximation ratio
 * F_p / C_max (Sec. 2). */
int64_t oracle_max_cut(int n, int m, const int32_t *edges, uint64_t *argmax)
{
    int64_t best = -1;
    uint64_t arg = 0;
    for (uint64_t x = 0; x < ((uint64_t)1 << n); x++) {
        int64_t c = oracle_cut_value(m, edges, x);
        if (c > best) {
            best = c;
            arg = x;
        }
    }
    *argmax = arg;
    return best;
}

/* Inverse-CDF sampling of basis states from |psi|^2: with the cumulative sums
 * S(x) = sum_{y <= x} |psi_y|^2 taken in index order, u_k in [0, 1) selects
 * the smallest x with S(x) > u_k S(2^n - 1) (the last index if none). The
 * uniform numbers are inputs, so no generator is needed here. */
int oracle_sample(int n, const cplx *psi, int K, const double *u, uint64_t *x_out)
{
    const uint64_t N = (uint64_t)1 << n;
    double *cdf = (double *)malloc(N * sizeof(double));
    if (!cdf)
        return -1;
    double s = 0.0;
    for (uint64_t x = 0; x < N; x++) {
        double a = creal(psi[x]), b = cimag(psi[x]);
        s += a * a + b * b;
        cdf[x] = s;
    }
    for (int k = 0; k < K; k++) {
        const double t = u[k] * s;
        uint64_t lo = 0, hi = N;  /* first x in [lo, hi) with cdf[x] > t */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > t)
                hi = mid;
            else
                lo = mid + 1;
        }
        x_out[k] = lo < N ? lo : N - 1;
    }
    free(cdf);
    return 0;
}

/* ------------------------------------------------------------------
 * Ising-form objectives (the generalisation named in the paper's
 * conclusion: weighted MaxCut and Ising objectives with fields):
 *   H = sum_e w_e 1/2 (1 - Z_u Z_v) + sum_i h_i 1/2 (1 - Z_i),
 * real w_e and h_i, whose diagonal is
 *   C(x) = sum_e w_e [x_u != x_v] + sum_i h_i x_i.
 * With every h_i = 0 and every w_e = 1 this is H_C of MaxCut. The same form
 * serves as the observable: H_red keeps one representative edge per edge
 * orbit at weight |orbit| w_rep and one representative vertex per vertex
 * orbit at weight |orbit| h_rep. h may be NULL (no fields). */
double oracle_ising_value(int m, const int32_t *edges, const double *w, int n, const double *h, uint64_t x)
{
    double s = 0.0;
    for (int e = 0; e < m; e++) {
        uint64_t xu = (x >> edges[2 * e]) & 1u, xv = (x >> edges[2 * e + 1]) & 1u;
        s += (xu != xv) ? w[e] : 0.0;
    }
    if (h)
        for (int i = 0; i < n; i++)
            if ((x >> i) & 1u)
                s += h[i];
    return s;
}

/* psi <- exp(-i gamma H) psi for the Ising-form H above. */
void oracle_ising_apply_cost(int n, int m, const int32_t *edges, const double *w, const double *h, double gamma,
                             cplx *psi)
{
    uint64_t N = 1ull << n;
#pragma omp parallel for
    for (uint64_t x = 0; x < N; x++)
        psi[x] *= cexp(-I * gamma * oracle_ising_value(m, edges, w, n, h, x));
}

/* The p-layer state of Eq. (1) with the Ising-form cost layer. */
void oracle_ising_state(int n, int m, const int32_t *edges, const double *w, const double *h, int p,
                        const double *gamma, const double *beta, cplx *psi)
{
    oracle_plus_state(n, psi);
    for (int l = 0; l < p; l++) {
        oracle_ising_apply_cost(n, m, edges, w, h, gamma[l], psi);
        oracle_apply_mixer(n, beta[l], psi);
    }
}

/* Energy <psi|O|psi> of an Ising-form observable O (edges ok, weights ow,
 * fields oh) and its gradient by the same adjoint recursion as
 * oracle_energy_grad, with the Ising-form cost as the generator of the
 * phase layers. Returns E. */
double oracle_ising_energy_grad(int n, int m, const int32_t *edges, const double *w, const double *h, int p,
                                const double *gamma, const double *beta, int k, const int32_t *oedges,
                                const double *ow, const double *oh, double *dgamma, double *dbeta, cplx *phi,
                                cplx *lam)
{
    uint64_t N = 1ull << n;
    oracle_ising_state(n, m, edges, w, h, p, gamma, beta, phi);
    double e_sum = 0.0;
#pragma omp parallel for reduction(+ : e_sum)
    for (uint64_t x = 0; x < N; x++) {
        double o = oracle_ising_value(k, oedges, ow, n, oh, x);
        lam[x] = o * phi[x];
        e_sum += o * (creal(phi[x]) * creal(phi[x]) + cimag(phi[x]) * cimag(phi[x]));
    }
    for (int l = p - 1; l >= 0; l--) {
        double im_sum = 0.0;
        for (int q = 0; q < n; q++) {
            uint64_t bit = 1ull << q;
#pragma omp parallel for reduction(+ : im_sum)
            for (uint64_t x = 0; x < N; x++)
                im_sum += cimag(conj(lam[x]) * phi[x ^ bit]);
        }
        dbeta[l] = 2.0 * im_sum;
        oracle_apply_mixer(n, -beta[l], phi);
        oracle_apply_mixer(n, -beta[l], lam);
        im_sum = 0.0;
#pragma omp parallel for reduction(+ : im_sum)
        for (uint64_t x = 0; x < N; x++)
            im_sum += cimag(conj(lam[x]) * oracle_ising_value(m, edges, w, n, h, x) * phi[x]);
        dgamma[l] = 2.0 * im_sum;
        oracle_ising_apply_cost(n, m, edges, w, h, -gamma[l], phi);
        oracle_ising_apply_cost(n, m, edges, w, h, -gamma[l], lam);
    }
    return e_sum;
}

/* Threads the loops above run on: 1 unless built with OpenMP. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
