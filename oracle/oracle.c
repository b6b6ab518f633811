/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for the QAOA hot path of
 * "Fast Simulation of High-Depth QAOA Circuits" (arXiv 2309.04841).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load or call this code.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * links or loads it.
 *
 * Every routine follows the paper's definitions literally, in complex128 /
 * float64 (int64 for integer costs), with no blocking, fusion or reordering:
 *   - cost polynomial over spins ............ Eq. 1 (Background)
 *   - MaxCut and LABS costs ................. Background section
 *   - phase operator (elementwise) .......... Sec. 3.1, Algorithm 3
 *   - single-qubit SU(2) update ............. Algorithm 1
 *   - uniform SU(2) transform (the mixer) ... Algorithm 2, Sec. 3.2
 *   - QAOA simulation ....................... Algorithm 3
 *   - expectation / ground-state overlap .... Sec. 3.1 (inner product), Sec. 4
 *   - XY mixers (ring, complete graph) ...... Sec. 3.2 (SU(4) extension of
 *     Algorithms 1-2), as the ordered product of the edge gates
 *   - adjoint gradient ...................... not in the paper; textbook
 *     reverse-mode differentiation of Algorithm 3 that keeps every
 *     intermediate state.
 *
 * Conventions (readings of the paper where it is silent or inconsistent):
 *   - qubit q (0-based) is bit q of the basis index x (least significant bit
 *     = qubit 0), which is Algorithm 1 with d = q + 1;
 *   - spin s_q(x) = +1 when bit q is 0 and -1 when it is 1;
 *   - the mixer gate is exp(-i beta X) = cos(beta) I - i sin(beta) X, i.e.
 *     Algorithm 1 with a = cos(beta), b = -i sin(beta) (Sec. 3.2 text; the
 *     "b = sin(beta)" printed in Algorithm 3 would give exp(-i beta Y));
 *   - the circuit is prod_l exp(-i beta_l M) exp(-i gamma_l C) applied to
 *     |+>^n (Background).
 *
 * Pinned by tests/test_oracle.py against closed forms, dense brute force,
 * identities and hand-checked small cases (never against the CUDA path).
 *
 * The elementwise loops carry OpenMP pragmas, which the oracle build
 * ignores (single thread).  A second build of this same source with
 * -fopenmp spreads those loops over the host cores for the benchmark's
 * all-core CPU figure; every element is still computed by the same
 * expression and the sums stay serial and pairwise, so both builds return
 * bit-identical results.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Spin of variable q in basis state x (Eq. 1: B = {-1, 1}). */
static int spin(uint64_t x, int q)
{
    return ((x >> q) & 1u) ? -1 : 1;
}

/* ------------------------------------------------------------------ costs */

/*
 * Eq. 1: f(s) = sum_k w_k prod_{i in t_k} s_i, integer weights, exact int64.
 * Terms are given in CSR form: term k uses indices tidx[tptr[k] .. tptr[k+1]).
 * An empty index set is the constant offset.
 */
void oracle_costs_terms_i64(int n, int n_terms, const int64_t *w,
                            const int32_t *tptr, const int32_t *tidx,
                            int64_t *f)
{
    uint64_t N = (uint64_t)1 << n;
    for (uint64_t x = 0; x < N; ++x) {
        int64_t acc = 0;
        for (int k = 0; k < n_terms; ++k) {
            int prod = 1;
            for (int j = tptr[k]; j < tptr[k + 1]; ++j)
                prod *= spin(x, tidx[j]);
            acc += w[k] * prod;
        }
        f[x] = acc;
    }
}

/* Eq. 1 with real weights, accumulated in float64 in term order. */
void oracle_costs_terms_f64(int n, int n_terms, const double *w,
                            const int32_t *tptr, const int32_t *tidx,
                            double *f)
{
    uint64_t N = (uint64_t)1 << n;
    for (uint64_t x = 0; x < N; ++x) {
        double acc = 0.0;
        for (int k = 0; k < n_terms; ++k) {
            int prod = 1;
            for (int j = tptr[k]; j < tptr[k + 1]; ++j)
                prod *= spin(x, tidx[j]);
            acc += w[k] * (double)prod;
        }
        f[x] = acc;
    }
}

/*
 * LABS energy of one sequence: f = sum_{k=1}^{n-1} C_k^2 with the aperiodic
 * autocorrelation C_k = sum_{i=0}^{n-k-1} s_i s_{i+k}.  This is the
 * sum-of-squares form; the paper's reduced 4-body/2-body polynomial
 * (Background) equals (f - n(n-1)/2) / 2.
 */
int64_t oracle_labs_cost_at(int n, uint64_t x)
{
    int64_t f = 0;
    for (int k = 1; k < n; ++k) {
        int64_t c = 0;
        for (int i = 0; i + k < n; ++i)
            c += spin(x, i) * spin(x, i + k);
        f += c * c;
    }
    return f;
}

void oracle_labs_costs(int n, int64_t *f)
{
    uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x)
        f[x] = oracle_labs_cost_at(n, x);
}

/* LABS energies for a contiguous index range [x0, x1), for sampled checks. */
void oracle_labs_costs_range(int n, uint64_t x0, uint64_t x1, int64_t *f)
{
    for (uint64_t x = x0; x < x1; ++x)
        f[x - x0] = oracle_labs_cost_at(n, x);
}

/*
 * Weighted MaxCut (Background, generalised to weights):
 * f = sum_{(i,j) in E} (w_ij / 2) (s_i s_j - 1), i.e. minus the weight of the
 * cut, accumulated in float64 in edge order.  edges holds m pairs (i, j).
 */
void oracle_maxcut_costs(int n, int m, const int32_t *edges, const double *w,
                         double *f)
{
    uint64_t N = (uint64_t)1 << n;
    for (uint64_t x = 0; x < N; ++x) {
        double acc = 0.0;
        for (int e = 0; e < m; ++e) {
            int si = spin(x, edges[2 * e]);
            int sj = spin(x, edges[2 * e + 1]);
            acc += 0.5 * w[e] * (double)(si * sj - 1);
        }
        f[x] = acc;
    }
}

/* ----------------------------------------------------------- simulation */

/* Uniform superposition |+>^n: every amplitude 2^{-n/2} (Background). */
void oracle_init_plus(int n, cplx *psi)
{
    uint64_t N = (uint64_t)1 << n;
    double a = 1.0 / sqrt((double)N);
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x)
        psi[x] = a;
}

/* Phase operator (Algorithm 3, step "apply phase operator"):
 * y_k <- exp(-i gamma c_k) y_k, with float64 cos/sin of the unreduced angle. */
void oracle_apply_phase(int n, cplx *psi, const double *f, double gamma)
{
    uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x) {
        double th = gamma * f[x];
        psi[x] *= cos(th) - I * sin(th);
    }
}

/*
 * Algorithm 1: apply U = [[a, -conj(b)], [b, conj(a)]] to qubit d (1-based),
 * in place.  In 0-based indices the paired elements are
 * l1 = k1 * 2^d + k2 and l2 = l1 + 2^{d-1}, k1 < 2^{n-d}, k2 < 2^{d-1}.
 */
static void apply_su2(int n, cplx *y, int d, cplx a, cplx b)
{
    uint64_t outer = (uint64_t)1 << (n - d);
    uint64_t half = (uint64_t)1 << (d - 1);
#pragma omp parallel for collapse(2) schedule(static)
    for (uint64_t k1 = 0; k1 < outer; ++k1) {
        for (uint64_t k2 = 0; k2 < half; ++k2) {
            uint64_t l1 = k1 * (half << 1) + k2;
            uint64_t l2 = l1 + half;
            cplx y1 = y[l1], y2 = y[l2];
            y[l1] = a * y1 - conj(b) * y2;
            y[l2] = b * y1 + conj(a) * y2;
        }
    }
}

/* Algorithm 1 with a = ar + i ai, b = br + i bi (plain doubles at the ABI). */
void oracle_apply_su2(int n, cplx *y, int d, double ar, double ai, double br,
                      double bi)
{
    apply_su2(n, y, d, ar + I * ai, br + I * bi);
}

/* Algorithm 2 with every U_i = exp(-i beta X): the transverse-field mixer
 * exp(-i beta sum_i X_i) (Sec. 3.2). */
void oracle_apply_mixer(int n, cplx *psi, double beta)
{
    cplx a = cos(beta);
    cplx b = -I * sin(beta);
    for (int d = 1; d <= n; ++d)
        apply_su2(n, psi, d, a, b);
}

/* Algorithm 3: p layers of phase then mixer.  If init_plus is nonzero the
 * state is first set to |+>^n, otherwise psi holds the input state. */
void oracle_simulate(int n, const double *f, int p, const double *gammas,
                     const double *betas, cplx *psi, int init_plus)
{
    if (init_plus)
        oracle_init_plus(n, psi);
    for (int l = 0; l < p; ++l) {
        oracle_apply_phase(n, psi, f, gammas[l]);
        oracle_apply_mixer(n, psi, betas[l]);
    }
}

/* ------------------------------------------------------------ XY mixers */

/*
 * exp(-i beta (X_i X_j + Y_i Y_j) / 2) on qubits i != j, in place (Sec. 3.2,
 * the SU(4) extension of Algorithm 1).  (XX + YY) / 2 swaps the two basis
 * states whose bits i, j are 01 and 10 and annihilates 00 and 11, so the gate
 * is the identity on the latter and [[cos b, -i sin b], [-i sin b, cos b]] on
 * each pair of states that differ exactly in bits i and j.
 */
void oracle_apply_xy(int n, cplx *psi, int i, int j, double beta)
{
    uint64_t N = (uint64_t)1 << n, mi = (uint64_t)1 << i, mj = (uint64_t)1 << j;
    cplx c = cos(beta), s = -I * sin(beta);
    for (uint64_t x = 0; x < N; ++x) {
        if ((x & mi) && !(x & mj)) {
            uint64_t y = x ^ mi ^ mj;
            cplx a = psi[x], b = psi[y];
            psi[x] = c * a + s * b;
            psi[y] = s * a + c * b;
        }
    }
}

/*
 * XY mixer of a graph on the n qubits: the product of the edge gates, the
 * first edge applied first.  graph 1 = ring: (0,1), (1,2), ..., (n-2,n-1),
 * then (n-1,0) when n >= 3; graph 2 = complete: (i,j), i < j, in
 * lexicographic order.  (The paper names the graphs, not the order.)
 */
void oracle_apply_xy_mixer(int n, cplx *psi, int graph, double beta)
{
    if (graph == 1) {
        for (int q = 0; q + 1 < n; ++q)
            oracle_apply_xy(n, psi, q, q + 1, beta);
        if (n >= 3)
            oracle_apply_xy(n, psi, n - 1, 0, beta);
    } else {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                oracle_apply_xy(n, psi, i, j, beta);
    }
}

/* Algorithm 3 with the XY mixer, from the state in psi (no |+> start: the XY
 * mixer keeps the Hamming weight, so the caller picks the sector). */
void oracle_simulate_xy(int n, const double *f, int p, const double *gammas,
                        const double *betas, cplx *psi, int graph)
{
    for (int l = 0; l < p; ++l) {
        oracle_apply_phase(n, psi, f, gammas[l]);
        oracle_apply_xy_mixer(n, psi, graph, betas[l]);
    }
}

/* Dicke state |D^n_k>: the uniform superposition of the C(n, k) basis
 * states of Hamming weight k. */
void oracle_dicke(int n, int k, cplx *psi)
{
    uint64_t N = (uint64_t)1 << n, cnt = 0;
    for (uint64_t x = 0; x < N; ++x)
        if (__builtin_popcountll(x) == k)
            ++cnt;
    double a = cnt ? 1.0 / sqrt((double)cnt) : 0.0;
    for (uint64_t x = 0; x < N; ++x)
        psi[x] = __builtin_popcountll(x) == k ? a : 0.0;
}

/* Pairwise (recursive halving) sum of v[0..len). */
static double pairwise_sum(const double *v, uint64_t len)
{
    if (len <= 8) {
        double s = 0.0;
        for (uint64_t i = 0; i < len; ++i)
            s += v[i];
        return s;
    }
    uint64_t h = len / 2;
    return pairwise_sum(v, h) + pairwise_sum(v + h, len - h);
}

/* Expectation <psi| diag(f) |psi> = sum_x |psi_x|^2 f_x (Sec. 3.1). */
double oracle_energy(int n, const cplx *psi, const double *f)
{
    uint64_t N = (uint64_t)1 << n;
    double *t = (double *)malloc(N * sizeof(double));
    if (!t)
        return NAN;
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x) {
        double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        t[x] = pr * f[x];
    }
    double s = pairwise_sum(t, N);
    free(t);
    return s;
}

/* Ground-state overlap: total probability of every x with f_x = min f
 * (Sec. 4, get_overlap with the cost vector as the default). */
double oracle_overlap(int n, const cplx *psi, const double *f)
{
    uint64_t N = (uint64_t)1 << n;
    double fmin = f[0];
    for (uint64_t x = 1; x < N; ++x)
        if (f[x] < fmin)
            fmin = f[x];
    double *t = (double *)malloc(N * sizeof(double));
    if (!t)
        return NAN;
    for (uint64_t x = 0; x < N; ++x) {
        double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        t[x] = (f[x] == fmin) ? pr : 0.0;
    }
    double s = pairwise_sum(t, N);
    free(t);
    return s;
}

/* Im <u|v> summed pairwise. */
static double im_inner(uint64_t N, const cplx *u, const cplx *v, double *tmp)
{
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x)
        tmp[x] = cimag(conj(u[x]) * v[x]);
    return pairwise_sum(tmp, N);
}

/*
 * Objective and its gradient with respect to every gamma_l and beta_l
 * (not in the paper).  Reverse-mode differentiation of Algorithm 3 that keeps
 * every intermediate state:
 *   phi_l = P(gamma_l) psi_{l-1},  psi_l = M(beta_l) phi_l,  E = <psi_p|F|psi_p>
 *   lam = F psi_p;  for l = p..1:
 *     dE/dbeta_l  = 2 Im <lam| B psi_l>,  B = sum_q X_q;   lam <- M(beta_l)^dag lam
 *     dE/dgamma_l = 2 Im <lam| F phi_l>;                   lam <- P(gamma_l)^dag lam
 * Returns 0 on success, -1 if memory could not be allocated.
 */
int oracle_grad(int n, const double *f, int p, const double *gammas,
                const double *betas, double *energy, double *dgamma,
                double *dbeta)
{
    uint64_t N = (uint64_t)1 << n;
    cplx *psi = (cplx *)malloc((size_t)(p + 1) * N * sizeof(cplx)); /* psi_0..psi_p */
    cplx *phi = (cplx *)malloc((size_t)(p + 1) * N * sizeof(cplx)); /* phi_1..phi_p */
    cplx *lam = (cplx *)malloc(N * sizeof(cplx));
    cplx *tmp = (cplx *)malloc(N * sizeof(cplx));
    double *rt = (double *)malloc(N * sizeof(double));
    if (!psi || !phi || !lam || !tmp || !rt) {
        free(psi); free(phi); free(lam); free(tmp); free(rt);
        return -1;
    }
    oracle_init_plus(n, psi);
    for (int l = 1; l <= p; ++l) {
        memcpy(phi + (size_t)l * N, psi + (size_t)(l - 1) * N, N * sizeof(cplx));
        oracle_apply_phase(n, phi + (size_t)l * N, f, gammas[l - 1]);
        memcpy(psi + (size_t)l * N, phi + (size_t)l * N, N * sizeof(cplx));
        oracle_apply_mixer(n, psi + (size_t)l * N, betas[l - 1]);
    }
    const cplx *psip = psi + (size_t)p * N;
    *energy = oracle_energy(n, psip, f);
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; ++x)
        lam[x] = f[x] * psip[x];
    for (int l = p; l >= 1; --l) {
        const cplx *psil = psi + (size_t)l * N;
        const cplx *phil = phi + (size_t)l * N;
        /* tmp = B psi_l = sum_q X_q psi_l, with (X_q v)[x] = v[x xor 2^q] */
#pragma omp parallel for schedule(static)
        for (uint64_t x = 0; x < N; ++x) {
            cplx s = 0.0;
            for (int q = 0; q < n; ++q)
                s += psil[x ^ ((uint64_t)1 << q)];
            tmp[x] = s;
        }
        dbeta[l - 1] = 2.0 * im_inner(N, lam, tmp, rt);
        oracle_apply_mixer(n, lam, -betas[l - 1]);
#pragma omp parallel for schedule(static)
        for (uint64_t x = 0; x < N; ++x)
            tmp[x] = f[x] * phil[x];
        dgamma[l - 1] = 2.0 * im_inner(N, lam, tmp, rt);
        oracle_apply_phase(n, lam, f, -gammas[l - 1]);
    }
    free(psi); free(phi); free(lam); free(tmp); free(rt);
    return 0;
}
