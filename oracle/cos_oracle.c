/*
 * CPU oracle for combinatorial-summation (CoS) graph evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * GPU path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the library never does.  It shares
 * no code, header or table with the CUDA path.
 *
 * What it computes (Sec. II.B and the caption of Fig. 1):
 *   - the top node of the leveled digraph holds 1;
 *   - each edge multiplies the value of its origin node by a propagator and
 *     adds the product to its destination node;
 *   - each node is the sum over its incoming edges;
 *   - the last node holds the sum over all root-to-sink paths (diagrams).
 * Edges are processed level by level in input order (the flattened layout of
 * Fig. 3: all edges of level 1, then level 2, ...), so every parent is final
 * before any of its out-edges is used (Sec. II.C, "Windowing").
 *
 * The edge factor is the free-fermion propagator of the synthetic workload,
 *   G_k(tau) = -exp(-eps_k tau) / (1 + exp(-beta eps_k))        0 <= tau < beta
 *   G_k(tau) = -G_k(tau + beta)                                 -beta < tau < 0
 * with tau = t_i - t_j formed in double precision; tau == 0 takes the first
 * branch.  The paper writes no formula for G (Fig. 1 caption only names the
 * Green's function G_ab), so this definition is the workload's.
 *
 * An edge whose kind field has bit 30 set closes a fermion loop: its factor is
 * additionally multiplied by -1 (Sec. II.C, "Numerical stability": the edge
 * operation checks whether the result must be multiplied by -1).  Bits 0..29 hold
 * the kind.
 *
 * Arithmetic is IEEE double with no contraction (build with -ffp-contract=off)
 * so results are the same on every host.  Path counts use 128-bit integers and
 * report overflow past 2^63-1; the int64 result wraps modulo 2^64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Free-fermion propagator G_k(tau) for one kind (eps) at inverse temperature beta. */
double cos_oracle_propagator(double eps, double beta, double tau) {
    if (tau >= 0.0) {
        return -exp(-eps * tau) / (1.0 + exp(-beta * eps));
    }
    /* antiperiodic continuation: G(tau) = -G(tau + beta) for -beta < tau < 0 */
    double shifted = tau + beta;
    return exp(-eps * shifted) / (1.0 + exp(-beta * eps));
}

void cos_oracle_propagator_array(double eps, double beta, const double* tau, double* out, int64_t n) {
    for (int64_t q = 0; q < n; ++q) out[q] = cos_oracle_propagator(eps, beta, tau[q]);
}

#define COS_ORACLE_SIGN_BIT 0x40000000
#define COS_ORACLE_KIND_MASK 0x3fffffff

static int check_graph(int32_t L, const int64_t* widths, const int64_t* counts, const int32_t* edges,
                       int32_t K, int32_t D, int64_t* N_out, int64_t* E_out) {
    if (L < 2) return -1;
    int64_t N = 0, E = 0;
    for (int32_t l = 0; l < L; ++l) { if (widths[l] < 1) return -1; N += widths[l]; E += counts[l]; }
    if (counts[0] != 0) return -1;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* r = edges + 5 * e;
        if (r[0] < 0 || r[0] >= N || r[1] < 0 || r[1] >= N) return -1;
        if (r[2] < 0 || (K > 0 && (r[2] & COS_ORACLE_KIND_MASK) >= K)) return -1;
        if (D > 0 && (r[3] < 0 || r[3] >= D || r[4] < 0 || r[4] >= D)) return -1;
    }
    *N_out = N; *E_out = E;
    return 0;
}

/* Level-wise dynamic program with given per-edge weights w[E] (sample-independent).
 * node_values[N] receives every node's value; node_values[N-1] is the path sum. */
int cos_oracle_pathsum(int32_t L, const int64_t* widths, const int64_t* counts, const int32_t* edges,
                       const double* w, double* node_values) {
    int64_t N, E;
    if (check_graph(L, widths, counts, edges, 0, 0, &N, &E)) return -1;
    for (int64_t n = 0; n < N; ++n) node_values[n] = 0.0;
    node_values[0] = 1.0;                       /* the top node holds 1 */
    for (int64_t e = 0; e < E; ++e) {           /* level-major input order */
        const int32_t* r = edges + 5 * e;
        node_values[r[1]] += node_values[r[0]] * w[e];
    }
    return 0;
}

/* Per-sample evaluation: R[s] = sink value with w_e = G_{k_e}(t_{s,i_e} - t_{s,j_e});
 * A[s] (optional) = the same DP with |w_e|, i.e. the sum of |path| values.
 * t is row-major [S][D]. */
int cos_oracle_eval(int32_t L, const int64_t* widths, const int64_t* counts, const int32_t* edges,
                    int32_t K, int32_t D, const double* eps, double beta,
                    int64_t S, const double* t, double* R, double* A, int32_t nthreads) {
    int64_t N, E;
    if (check_graph(L, widths, counts, edges, K, D, &N, &E)) return -1;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double* v = (double*)malloc(sizeof(double) * (size_t)N);
        double* a = A ? (double*)malloc(sizeof(double) * (size_t)N) : NULL;
        if (!v || (A && !a)) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t s = 0; s < S; ++s) {
                const double* ts = t + s * D;
                for (int64_t n = 0; n < N; ++n) v[n] = 0.0;
                v[0] = 1.0;
                if (a) { for (int64_t n = 0; n < N; ++n) a[n] = 0.0; a[0] = 1.0; }
                for (int64_t e = 0; e < E; ++e) {
                    const int32_t* r = edges + 5 * e;
                    double tau = ts[r[3]] - ts[r[4]];
                    double w = cos_oracle_propagator(eps[r[2] & COS_ORACLE_KIND_MASK], beta, tau);
                    if (r[2] & COS_ORACLE_SIGN_BIT) w = -w;   /* closes a fermion loop */
                    v[r[1]] += v[r[0]] * w;
                    if (a) a[r[1]] += a[r[0]] * fabs(w);
                }
                R[s] = v[N - 1];
                if (a) A[s] = a[N - 1];
            }
        }
        free(v);
        free(a);
    }
    return status;
}

/* The same evaluation carried in long double (the host's extended format: 64-bit
 * significand on x86-64, IEEE binary128 on AArch64) with expl: a reference whose
 * rounding error is far below double's, against which the double results (here
 * and on the GPU) can be measured.  tau = t_i - t_j is formed in long double from
 * the double times; the branch is still decided by t_i >= t_j on the doubles.
 * R[s] is the long double sink value rounded once to double. */
static long double propagator_ld(long double eps, long double beta, double ti, double tj) {
    const long double tau = (long double)ti - (long double)tj;
    if (ti >= tj) return -expl(-eps * tau) / (1.0L + expl(-beta * eps));
    return expl(-eps * (tau + beta)) / (1.0L + expl(-beta * eps));
}

int cos_oracle_eval_ld(int32_t L, const int64_t* widths, const int64_t* counts, const int32_t* edges,
                       int32_t K, int32_t D, const double* eps, double beta,
                       int64_t S, const double* t, double* R, int32_t nthreads) {
    int64_t N, E;
    if (check_graph(L, widths, counts, edges, K, D, &N, &E)) return -1;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        long double* v = (long double*)malloc(sizeof(long double) * (size_t)N);
        if (!v) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t s = 0; s < S; ++s) {
                const double* ts = t + s * D;
                for (int64_t n = 0; n < N; ++n) v[n] = 0.0L;
                v[0] = 1.0L;
                for (int64_t e = 0; e < E; ++e) {
                    const int32_t* r = edges + 5 * e;
                    long double w = propagator_ld((long double)eps[r[2] & COS_ORACLE_KIND_MASK], (long double)beta,
                                                  ts[r[3]], ts[r[4]]);
                    if (r[2] & COS_ORACLE_SIGN_BIT) w = -w;
                    v[r[1]] += v[r[0]] * w;
                }
                R[s] = (double)v[N - 1];
            }
        }
        free(v);
    }
    return status;
}

/* Unit-weight path count.  *count_wrapped = count mod 2^64 (as int64);
 * *overflow = 1 if the exact count exceeds 2^63-1. */
int cos_oracle_count(int32_t L, const int64_t* widths, const int64_t* counts, const int32_t* edges,
                     int64_t* count_wrapped, int32_t* overflow) {
    int64_t N, E;
    if (check_graph(L, widths, counts, edges, 0, 0, &N, &E)) return -1;
    uint64_t* wrap = (uint64_t*)calloc((size_t)N, sizeof(uint64_t));
    unsigned __int128* exact = (unsigned __int128*)calloc((size_t)N, sizeof(unsigned __int128));
    if (!wrap || !exact) { free(wrap); free(exact); return -2; }
    const unsigned __int128 cap = ((unsigned __int128)1) << 120;   /* saturate well below 2^128 */
    wrap[0] = 1; exact[0] = 1;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* r = edges + 5 * e;
        wrap[r[1]] += wrap[r[0]];
        unsigned __int128 x = exact[r[1]] + exact[r[0]];
        exact[r[1]] = x > cap ? cap : x;
    }
    *count_wrapped = (int64_t)wrap[N - 1];
    *overflow = exact[N - 1] > (unsigned __int128)INT64_MAX ? 1 : 0;
    free(wrap);
    free(exact);
    return 0;
}

/* Neumaier-compensated sum of x[0..n) in index order. */
double cos_oracle_neumaier_sum(const double* x, int64_t n) {
    double sum = 0.0, c = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        double y = x[q];
        double u = sum + y;
        if (fabs(sum) >= fabs(y)) c += (sum - u) + y;
        else c += (y - u) + sum;
        sum = u;
    }
    return sum + c;
}
