/*
 * ifctn_oracle.c -- plain, slow, FP64 CPU oracle of iFCTN tensor completion.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * GPU library: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes (paper: "iFCTN: an intra-block Fully-Connected Tensor
 * Network Decomposition for Tensor Completion", Gan & Cui):
 *
 *   - eq. (iFCTN), Def. 2: the element-wise iFCTN model.  The sum over every
 *     rank index r_{k,l} factorises pair by pair, because r_{k,l} occurs only
 *     in G_{k,l}(., i_k) and G_{l,k}(., i_l); so
 *         X(i) = prod_{k<l} W_{k,l}(i_k, i_l),  W_{k,l} = G_{k,l}^T G_{l,k}.
 *     This is the broadcast-Hadamard product that Prop. 1 calls S_k, taken
 *     over all pairs.
 *   - Sec. 4.2, eq. (updateG): one proximal block update per column j of
 *     G_{k,i}.  The coefficient row for tensor entry i (with i_k = j) is
 *         a(r) = T(i) * G_{i,k}(r, i_i),
 *         T(i) = prod over all pairs (p,q) other than {k,i} of W_{p,q}(i_p,i_q),
 *     which is D (y_j kron G_{i,k}^T) written entry by entry.  The normal
 *     equations are (A^T A + rho I) g = A^T x_j + rho g_old, solved by a
 *     textbook Cholesky factorisation.
 *   - Sec. 4.2, eq. (updateX): X <- P_{Omega^c}((iFCTN(G) + rho X)/(1+rho))
 *     + P_Omega(O); observed entries are left as they are.
 *   - Algorithm 1: blocks in the order k = 1..N, i != k ascending, every block
 *     using the latest value of every other factor (Gauss-Seidel), X^{(s)} held
 *     fixed for all factor blocks of sweep s; stop when
 *     ||X^{s+1}-X^s||_F / ||X^s||_F < eps or after t_max sweeps.
 *
 * Readings where the paper is silent or garbled:
 *   - fit term weighted 1/2 (as the closed form and Lemma 2 imply);
 *   - X^0 = P_Omega(O), zero elsewhere;
 *   - RSE = ||X_true - X|| / ||X_true||, RMSE over the missing entries.
 *
 * Layout.  Tensors are C order (last index fastest), 0-based.  Factor
 * G_{k,l} (l != k) is an R_{k,l} x I_k row-major block; blocks are packed in
 * the order k = 0..N-1, then l = 0..N-1 (l != k).  The rank matrix is a 4x4
 * row-major int array R[k*4+l], symmetric, diagonal ignored.
 *
 * Sums are Neumaier-compensated so the oracle's own rounding error stays
 * near 1e-16 relative.  Threads (OpenMP) split only independent columns j
 * and fixed element blocks; every reduction runs in a fixed order, so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IFO_MAXN 4
#define IFO_RMAX 64 /* largest R_{k,l}: the block buffers below are sized for it */

/* ------------------------------------------------------------------ */
/* compensated summation                                               */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;

static inline void kadd(ksum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double kval(const ksum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* shape helpers                                                       */
/* ------------------------------------------------------------------ */
static int rank_of(const int32_t* R, int k, int l) { return R[k * 4 + l]; }

long long ifo_numel(int N, const int64_t* dims) {
    long long P = 1;
    for (int k = 0; k < N; ++k) P *= dims[k];
    return P;
}

/* element offset of block G_{k,l} inside the packed factor array */
long long ifo_factor_offset(int N, const int64_t* dims, const int32_t* R, int k, int l) {
    long long off = 0;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            if (a == b) continue;
            if (a == k && b == l) return off;
            off += (long long)rank_of(R, a, b) * dims[a];
        }
    return -1;
}

/* number of parameters: sum_k I_k sum_{l != k} R_{k,l}  (Sec. 4.3, Table 5) */
long long ifo_param_count(int N, const int64_t* dims, const int32_t* R) {
    long long n = 0;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l)
            if (l != k) n += (long long)rank_of(R, k, l) * dims[k];
    return n;
}

static void c_strides(int N, const int64_t* dims, long long* st) {
    st[N - 1] = 1;
    for (int k = N - 2; k >= 0; --k) st[k] = st[k + 1] * dims[k + 1];
}

/* W_{p,q}(a,b) = sum_r G_{p,q}(r,a) G_{q,p}(r,b); p<q, I_p x I_q row-major.
   This is the matrix reshape(G_{p,q}^T G_{q,p}) of Prop. 1's S_k. */
void ifo_pair_matrix(int N, const int64_t* dims, const int32_t* R, const double* G,
                     int p, int q, double* W) {
    const int Rpq = rank_of(R, p, q);
    const double* Gpq = G + ifo_factor_offset(N, dims, R, p, q);
    const double* Gqp = G + ifo_factor_offset(N, dims, R, q, p);
    const long long Ip = dims[p], Iq = dims[q];
    for (long long a = 0; a < Ip; ++a)
        for (long long b = 0; b < Iq; ++b) {
            ksum s = {0, 0};
            for (int r = 0; r < Rpq; ++r) kadd(&s, Gpq[r * Ip + a] * Gqp[r * Iq + b]);
            W[a * Iq + b] = kval(&s);
        }
}

/* all pair matrices, stored in a [4][4] table of pointers (p<q) */
typedef struct { double* w[IFO_MAXN][IFO_MAXN]; } pairset;

static int pairs_alloc(int N, const int64_t* dims, pairset* ps) {
    memset(ps, 0, sizeof(*ps));
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) {
            ps->w[p][q] = (double*)malloc(sizeof(double) * dims[p] * dims[q]);
            if (!ps->w[p][q]) return -1;
        }
    return 0;
}
static void pairs_free(int N, pairset* ps) {
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) free(ps->w[p][q]);
}
static void pairs_compute(int N, const int64_t* dims, const int32_t* R, const double* G, pairset* ps) {
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) ifo_pair_matrix(N, dims, R, G, p, q, ps->w[p][q]);
}
static inline double wlook(const pairset* ps, const int64_t* dims, int p, int q, const long long* idx) {
    /* W_{p,q}(i_p, i_q) for p<q */
    return ps->w[p][q][idx[p] * dims[q] + idx[q]];
}

static void unflatten(int N, const int64_t* dims, long long e, long long* idx) {
    for (int k = N - 1; k >= 0; --k) { idx[k] = e % dims[k]; e /= dims[k]; }
}

/* ------------------------------------------------------------------ */
/* reconstruction, eq. (iFCTN)                                          */
/* ------------------------------------------------------------------ */
static double recon_at(int N, const int64_t* dims, const pairset* ps, const long long* idx) {
    double v = 1.0;
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) v *= wlook(ps, dims, p, q, idx);
    return v;
}

int ifo_reconstruct(int N, const int64_t* dims, const int32_t* R, const double* G, double* out) {
    if (N < 2 || N > IFO_MAXN) return -1;
    pairset ps;
    if (pairs_alloc(N, dims, &ps)) { pairs_free(N, &ps); return -2; }
    pairs_compute(N, dims, R, G, &ps);
    const long long P = ifo_numel(N, dims);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < P; ++e) {
        long long idx[IFO_MAXN];
        unflatten(N, dims, e, idx);
        out[e] = recon_at(N, dims, &ps, idx);
    }
    pairs_free(N, &ps);
    return 0;
}

/* ------------------------------------------------------------------ */
/* one proximal block: normal equations of column j of G_{k,i}          */
/* ------------------------------------------------------------------ */
/* Accumulates H = A^T A and b = A^T x for column j of G_{k,i}, where the row
   of A for entry i (i_k = j) is a(r) = T(i) G_{i,k}(r, i_i) and x is the
   mode-k slice X(i_k = j, :).  T multiplies every pair matrix except W_{k,i}.
   H is Rki x Rki (row-major), b has Rki entries.  Returns nonzero when the
   accumulators cannot be allocated. */
static int block_normal_eq(int N, const int64_t* dims, const int32_t* R, const double* G,
                           const pairset* ps, const double* X, int k, int i, long long j,
                           double* H, double* b) {
    const int Rki = rank_of(R, k, i);
    const double* Gik = G + ifo_factor_offset(N, dims, R, i, k);
    const long long Ii = dims[i];
    long long st[IFO_MAXN];
    c_strides(N, dims, st);
    /* lower triangle of H (row r, column c <= r at r(r+1)/2 + c) and b */
    ksum* hs = (ksum*)calloc((size_t)Rki * (Rki + 1) / 2 + Rki, sizeof(ksum));
    if (!hs) return 1;
    ksum* bs = hs + (size_t)Rki * (Rki + 1) / 2;
    /* odometer over all modes except k */
    long long idx[IFO_MAXN] = {0, 0, 0, 0};
    idx[k] = j;
    const long long Pk = ifo_numel(N, dims) / dims[k];
    double a[IFO_RMAX];
    for (long long t = 0; t < Pk; ++t) {
        double T = 1.0;
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) {
                if ((p == k && q == i) || (p == i && q == k)) continue;
                T *= wlook(ps, dims, p, q, idx);
            }
        long long flat = 0;
        for (int m = 0; m < N; ++m) flat += idx[m] * st[m];
        const double x = X[flat];
        for (int r = 0; r < Rki; ++r) a[r] = T * Gik[r * Ii + idx[i]];
        for (int r = 0; r < Rki; ++r) {
            kadd(&bs[r], a[r] * x);
            ksum* hr = hs + (size_t)r * (r + 1) / 2;
            for (int c = 0; c <= r; ++c) kadd(&hr[c], a[r] * a[c]);
        }
        /* advance the odometer (last mode fastest), skipping mode k */
        for (int m = N - 1; m >= 0; --m) {
            if (m == k) continue;
            if (++idx[m] < dims[m]) break;
            idx[m] = 0;
        }
    }
    for (int r = 0; r < Rki; ++r) {
        b[r] = kval(&bs[r]);
        for (int c = 0; c <= r; ++c) {
            H[r * Rki + c] = kval(&hs[(size_t)r * (r + 1) / 2 + c]);
            H[c * Rki + r] = H[r * Rki + c];
        }
    }
    free(hs);
    return 0;
}

/* Public: H = A^T A and b = A^T x (no proximal terms) for column j of G_{k,i}
   at the given state (G, X).  1 <= R_{k,i} <= IFO_RMAX. */
int ifo_block_system(int N, const int64_t* dims, const int32_t* R, const double* G,
                     const double* X, int k, int i, long long j, double* H, double* b) {
    if (N < 2 || N > IFO_MAXN || k == i || rank_of(R, k, i) < 1 || rank_of(R, k, i) > IFO_RMAX) return -1;
    pairset ps;
    if (pairs_alloc(N, dims, &ps)) { pairs_free(N, &ps); return -2; }
    pairs_compute(N, dims, R, G, &ps);
    const int rc = block_normal_eq(N, dims, R, G, &ps, X, k, i, j, H, b);
    pairs_free(N, &ps);
    return rc ? -2 : 0;
}

/* textbook Cholesky H = L L^T (lower, in place) and solve H g = rhs.
   Returns 0 on success, 1 if a pivot is not positive. */
int ifo_cholesky_solve(int n, double* H, double* rhs) {
    for (int c = 0; c < n; ++c) {
        double d = H[c * n + c];
        for (int t = 0; t < c; ++t) d -= H[c * n + t] * H[c * n + t];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        H[c * n + c] = d;
        for (int r = c + 1; r < n; ++r) {
            double v = H[r * n + c];
            for (int t = 0; t < c; ++t) v -= H[r * n + t] * H[c * n + t];
            H[r * n + c] = v / d;
        }
    }
    for (int r = 0; r < n; ++r) { /* forward: L y = rhs */
        double v = rhs[r];
        for (int t = 0; t < r; ++t) v -= H[r * n + t] * rhs[t];
        rhs[r] = v / H[r * n + r];
    }
    for (int r = n - 1; r >= 0; --r) { /* backward: L^T g = y */
        double v = rhs[r];
        for (int t = r + 1; t < n; ++t) v -= H[t * n + r] * rhs[t];
        rhs[r] = v / H[r * n + r];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* one PAM sweep (Algorithm 1, one pass of the while loop)             */
/* ------------------------------------------------------------------ */
/* stats[0] rel_change = ||X1-X0|| / ||X0||
   stats[1] objective  = 1/2 ||X1 - iFCTN(G1)||^2
   stats[2] rse        = ||Xt - X1|| / ||Xt||              (xtrue given, else NaN)
   stats[3] rmse       = sqrt(sum_{missing}(Xt-X1)^2 / #missing)  (else NaN)
   stats[4] ||X1-X0||^2, stats[5] ||X0||^2 */
#define IFO_BLOCK 65536

int ifo_sweep(int N, const int64_t* dims, const int32_t* R, double rho, double* G, double* X,
              const uint8_t* mask, const double* xtrue, int nthreads, double* stats) {
    if (N < 2 || N > IFO_MAXN || !(rho > 0.0)) return -1;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l)
            if (l != k && (rank_of(R, k, l) < 1 || rank_of(R, k, l) > IFO_RMAX ||
                           rank_of(R, k, l) != rank_of(R, l, k))) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    pairset ps;
    if (pairs_alloc(N, dims, &ps)) { pairs_free(N, &ps); return -2; }
    pairs_compute(N, dims, R, G, &ps);
    int bad = 0;
    /* factor blocks, eq. (updateG), in the order k, then i != k ascending */
    for (int k = 0; k < N; ++k) {
        for (int i = 0; i < N; ++i) {
            if (i == k) continue;
            const int Rki = rank_of(R, k, i);
            double* Gki = G + ifo_factor_offset(N, dims, R, k, i);
            const long long Ik = dims[k];
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
            for (long long j = 0; j < Ik; ++j) {
                double H[IFO_RMAX * IFO_RMAX], b[IFO_RMAX];
                if (block_normal_eq(N, dims, R, G, &ps, X, k, i, j, H, b)) { bad |= 2; continue; }
                for (int r = 0; r < Rki; ++r) {
                    H[r * Rki + r] += rho;
                    b[r] += rho * Gki[r * Ik + j];
                }
                if (ifo_cholesky_solve(Rki, H, b)) { bad |= 1; continue; }
                for (int r = 0; r < Rki; ++r) Gki[r * Ik + j] = b[r];
            }
            /* the pair matrix of {k,i} now uses the new G_{k,i} */
            const int p = k < i ? k : i, q = k < i ? i : k;
            ifo_pair_matrix(N, dims, R, G, p, q, ps.w[p][q]);
        }
    }
    /* X update, eq. (updateX), with fixed-block compensated reductions */
    const long long P = ifo_numel(N, dims);
    const long long nb = (P + IFO_BLOCK - 1) / IFO_BLOCK;
    double* part = (double*)calloc((size_t)nb * 6, sizeof(double));
    if (!part) { pairs_free(N, &ps); return -2; }
#pragma omp parallel for schedule(static)
    for (long long blk = 0; blk < nb; ++blk) {
        ksum dx = {0, 0}, x0 = {0, 0}, ob = {0, 0}, et = {0, 0}, tt = {0, 0}, em = {0, 0};
        long long nmiss = 0;
        const long long e0 = blk * IFO_BLOCK, e1 = e0 + IFO_BLOCK < P ? e0 + IFO_BLOCK : P;
        long long idx[IFO_MAXN];
        for (long long e = e0; e < e1; ++e) {
            unflatten(N, dims, e, idx);
            const double rec = recon_at(N, dims, &ps, idx);
            const double xo = X[e];
            const double xn = mask[e] ? xo : (rec + rho * xo) / (1.0 + rho);
            kadd(&dx, (xn - xo) * (xn - xo));
            kadd(&x0, xo * xo);
            kadd(&ob, (xn - rec) * (xn - rec));
            if (xtrue) {
                const double d = xtrue[e] - xn;
                kadd(&et, d * d);
                kadd(&tt, xtrue[e] * xtrue[e]);
                if (!mask[e]) { kadd(&em, d * d); ++nmiss; }
            }
            X[e] = xn;
        }
        double* pp = part + blk * 6;
        pp[0] = kval(&dx); pp[1] = kval(&x0); pp[2] = kval(&ob);
        pp[3] = kval(&et); pp[4] = kval(&tt); pp[5] = kval(&em);
        (void)nmiss;
    }
    ksum s[6];
    memset(s, 0, sizeof(s));
    for (long long blk = 0; blk < nb; ++blk)
        for (int t = 0; t < 6; ++t) kadd(&s[t], part[blk * 6 + t]);
    free(part);
    long long nmiss = 0;
    if (xtrue)
        for (long long e = 0; e < P; ++e) nmiss += mask[e] ? 0 : 1;
    const double dx2 = kval(&s[0]), x02 = kval(&s[1]);
    stats[0] = x02 > 0 ? sqrt(dx2) / sqrt(x02) : (dx2 > 0 ? INFINITY : 0.0);
    stats[1] = 0.5 * kval(&s[2]);
    if (xtrue) {
        const double t2 = kval(&s[4]);
        stats[2] = t2 > 0 ? sqrt(kval(&s[3])) / sqrt(t2) : NAN;
        stats[3] = nmiss > 0 ? sqrt(kval(&s[5]) / (double)nmiss) : 0.0;
    } else {
        stats[2] = NAN;
        stats[3] = NAN;
    }
    stats[4] = dx2;
    stats[5] = x02;
    pairs_free(N, &ps);
    return (bad & 2) ? -2 : (bad ? 1 : 0);
}

/* X^0 = P_Omega(O): observed values kept, zero elsewhere (Algorithm 1 init). */
void ifo_init_x(long long P, const double* O, const uint8_t* mask, double* X) {
    for (long long e = 0; e < P; ++e) X[e] = mask[e] ? O[e] : 0.0;
}

/* objective f(G, X) = 1/2 ||X - iFCTN(G)||^2 (Sec. 4.1) */
double ifo_objective(int N, const int64_t* dims, const int32_t* R, const double* G, const double* X) {
    pairset ps;
    if (pairs_alloc(N, dims, &ps)) { pairs_free(N, &ps); return NAN; }
    pairs_compute(N, dims, R, G, &ps);
    const long long P = ifo_numel(N, dims);
    ksum s = {0, 0};
    long long idx[IFO_MAXN];
    for (long long e = 0; e < P; ++e) {
        unflatten(N, dims, e, idx);
        const double d = X[e] - recon_at(N, dims, &ps, idx);
        kadd(&s, d * d);
    }
    pairs_free(N, &ps);
    return 0.5 * kval(&s);
}

/* Algorithm 1 from the given state (G, X): sweeps until the relative change
   drops below tol (tol > 0) or max_sweeps is reached.  stats_log receives
   6 doubles per sweep (see ifo_sweep).  Returns the sweep status. */
int ifo_complete(int N, const int64_t* dims, const int32_t* R, double rho, int max_sweeps,
                 double tol, double* G, double* X, const uint8_t* mask, const double* xtrue,
                 int nthreads, double* stats_log, int* sweeps_done) {
    int s = 0, rc = 0;
    for (; s < max_sweeps; ++s) {
        rc = ifo_sweep(N, dims, R, rho, G, X, mask, xtrue, nthreads, stats_log + 6 * s);
        if (rc) { ++s; break; }
        if (tol > 0 && stats_log[6 * s] < tol) { ++s; break; }
    }
    *sweeps_done = s;
    return rc;
}

/* Metrics of Sec. 5 on a given X: out[0] RSE = ||Xt - X|| / ||Xt||,
   out[1] RMSE = sqrt(sum over missing entries of (Xt - X)^2 / #missing). */
void ifo_metrics(long long P, const double* xtrue, const double* X, const uint8_t* mask,
                 double* out) {
    ksum e = {0, 0}, t = {0, 0}, m = {0, 0};
    long long nm = 0;
    for (long long i = 0; i < P; ++i) {
        const double d = xtrue[i] - X[i];
        kadd(&e, d * d);
        kadd(&t, xtrue[i] * xtrue[i]);
        if (!mask[i]) { kadd(&m, d * d); ++nm; }
    }
    out[0] = kval(&t) > 0 ? sqrt(kval(&e)) / sqrt(kval(&t)) : NAN;
    out[1] = nm > 0 ? sqrt(kval(&m) / (double)nm) : 0.0;
}
