/*
 * FP64 CPU oracle for the Monte-Carlo estimator of Pauli-Z expectation values
 * of parameterised IQP circuits (arxiv 2501.04776).
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and bench.py's
 * CPU baseline / reference arm may load or call this library. It shares no
 * code with the CUDA path and the CUDA path never calls it.
 *
 * Plain, slow and obviously correct: bits are read one qubit at a time, GF(2)
 * inner products are XORs over the support of a generator or observable, all
 * floating point is double precision, and every sum runs in natural index
 * order. Skipping a term that is exactly zero (a qubit outside the support,
 * a gate that commutes with the observable) leaves every sum bit-identical.
 *
 * Inputs use the bit format of the C ABI: a binary matrix is uint64 words,
 * row-major, `ld` words per row, LSB-first (bit b of word w is column 64w+b).
 *
 * What pins each function against the paper and the mathematics is in
 * tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int bit_at(const uint64_t *row, int64_t q) {
    return (int)((row[q >> 6] >> (q & 63)) & 1u);
}

/* Support (list of qubits with a 1) of every row of a packed matrix. */
typedef struct {
    int64_t *start; /* rows+1 offsets */
    int32_t *idx;
} support_t;

/* Words that are zero hold no qubit of the support and are skipped. */
static support_t support_of(const uint64_t *M, int64_t rows, int64_t ld, int64_t n) {
    support_t sp;
    const int64_t nw = (n + 63) / 64;
    sp.start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rows + 1));
    int64_t total = 0;
    for (int64_t r = 0; r < rows; ++r) {
        sp.start[r] = total;
        for (int64_t w = 0; w < nw; ++w) {
            if (M[r * ld + w] == 0) continue;
            for (int64_t q = 64 * w; q < 64 * w + 64 && q < n; ++q) total += bit_at(M + r * ld, q);
        }
    }
    sp.start[rows] = total;
    sp.idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t w = 0; w < nw; ++w) {
            if (M[r * ld + w] == 0) continue;
            for (int64_t q = 64 * w; q < 64 * w + 64 && q < n; ++q)
                if (bit_at(M + r * ld, q)) sp.idx[k++] = (int32_t)q;
        }
    return sp;
}

static void support_free(support_t *sp) {
    free(sp->start);
    free(sp->idx);
}

/* Unpack rows of a packed matrix to one byte per bit. */
static uint8_t *unpack_rows(const uint64_t *M, int64_t rows, int64_t ld, int64_t n) {
    uint8_t *b = (uint8_t *)malloc((size_t)(rows > 0 ? rows : 1) * (size_t)(n > 0 ? n : 1));
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t q = 0; q < n; ++q) b[r * n + q] = (uint8_t)bit_at(M + r * ld, q);
    return b;
}

/* GF(2) inner products of every row r of R with every generator g_j:
 * P[r*m + j] = (sum_q R[r][q] * G[j][q]) mod 2. With R = A this is A.G^T,
 * with R = Z it is Z.G^T (Sec. 2.2, definitions of B and C). */
static uint8_t *parity_matrix(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr,
                              const uint64_t *G, int64_t m, int64_t ldg) {
    uint8_t *Rb = unpack_rows(R, rows, ldr, n);
    support_t sg = support_of(G, m, ldg, n);
    uint8_t *P = (uint8_t *)malloc((size_t)(rows > 0 ? rows : 1) * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        const uint8_t *rb = Rb + r * n;
        for (int64_t j = 0; j < m; ++j) {
            int x = 0;
            for (int64_t k = sg.start[j]; k < sg.start[j + 1]; ++k) x ^= rb[sg.idx[k]];
            P[r * m + j] = (uint8_t)x;
        }
    }
    support_free(&sg);
    free(Rb);
    return P;
}

/* Public parity: P is rows x m bytes (0/1). */
void oracle_parity(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr,
                   const uint64_t *G, int64_t m, int64_t ldg, uint8_t *P) {
    uint8_t *p = parity_matrix(n, R, rows, ldr, G, m, ldg);
    memcpy(P, p, (size_t)rows * (size_t)m);
    free(p);
}

/* Gates that anticommute with observable a: J_a = { j : P_A[a][j] = 1 }.
 * Only these have C_{a,j} = 1 - (-1)^{a.g_j} = 2 (Sec. 2.2, matrix C). */
static int64_t gates_of(const uint8_t *PA_row, int64_t m, int64_t *J) {
    int64_t k = 0;
    for (int64_t j = 0; j < m; ++j)
        if (PA_row[j]) J[k++] = j;
    return k;
}

/* Phase of sample i for observable a (eq. expvalsample / Emat):
 * Phi = sum_j theta_j * (-1)^{g_j.z_i} * (1 - (-1)^{g_j.a}),
 * i.e. sum over J_a of 2 theta_j (1 - 2 P_Z[i][j]). */
static double phase(const int64_t *J, int64_t k, const double *theta, const uint8_t *PZ_row) {
    double phi = 0.0;
    for (int64_t t = 0; t < k; ++t) {
        int64_t j = J[t];
        double sign = PZ_row[j] ? -1.0 : 1.0;
        phi += theta[j] * sign * 2.0;
    }
    return phi;
}

/* Monte-Carlo estimate (eq. expvalsample) of <Z_a> for every observable,
 * with its standard error: population standard deviation of cos(Phi) over
 * the s samples (ddof = 0, two-pass), divided by sqrt(s). Also returns
 * S1 = sum_i cos(Phi) and S2 = sum_i cos(Phi)^2 (any output may be NULL). */
void oracle_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                   const uint64_t *A, int64_t l, int64_t lda,
                   const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                   double *expval, double *std_err, double *S1, double *S2) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    uint8_t *PZ = parity_matrix(n, Z, s, ldz, G, m, ldg);
#pragma omp parallel
    {
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        double *c = (double *)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
#pragma omp for schedule(static)
        for (int64_t a = 0; a < l; ++a) {
            int64_t k = gates_of(PA + a * m, m, J);
            double sum = 0.0, sum2 = 0.0;
            for (int64_t i = 0; i < s; ++i) {
                c[i] = cos(phase(J, k, theta, PZ + i * m));
                sum += c[i];
                sum2 += c[i] * c[i];
            }
            double mean = sum / (double)s;
            double dev2 = 0.0;
            for (int64_t i = 0; i < s; ++i) dev2 += (c[i] - mean) * (c[i] - mean);
            if (expval) expval[a] = mean;
            if (std_err) std_err[a] = sqrt(dev2 / (double)s) / sqrt((double)s);
            if (S1) S1[a] = sum;
            if (S2) S2[a] = sum2;
        }
        free(c);
        free(J);
    }
    free(PZ);
    free(PA);
}

/* Gradient of any loss whose derivative with respect to the estimator's
 * samples has the form  dL/dPhi[a][i] = -sin(Phi) (alpha_a + beta_a cos(Phi)):
 *   grad_j = sum_a sum_i sin(Phi[a][i]) (alpha_a + beta_a cos(Phi[a][i]))
 *                        * dPhi[a][i]/dtheta_j,
 *   dPhi[a][i]/dtheta_j = 2 P_A[a][j] (1 - 2 P_Z[i][j]).
 * For L = sum_a w_a <Z_a>^ pass alpha_a = -w_a/s, beta = NULL (Sec. 2.4: the
 * estimator is a deterministic, differentiable function of theta for fixed
 * samples). Accumulated per thread over a static split of observables and
 * summed in thread order. */
void oracle_expval_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                        const uint64_t *A, int64_t l, int64_t lda,
                        const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                        const double *alpha, const double *beta, double *grad) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    uint8_t *PZ = parity_matrix(n, Z, s, ldz, G, m, ldg);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *part = (double *)calloc((size_t)nthreads * (size_t)(m > 0 ? m : 1), sizeof(double));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *g = part + (size_t)tid * (size_t)m;
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(static)
        for (int64_t a = 0; a < l; ++a) {
            int64_t k = gates_of(PA + a * m, m, J);
            double al = alpha ? alpha[a] : 0.0, be = beta ? beta[a] : 0.0;
            for (int64_t i = 0; i < s; ++i) {
                const uint8_t *pz = PZ + i * m;
                double phi = phase(J, k, theta, pz);
                double w = sin(phi) * (al + be * cos(phi));
                for (int64_t t = 0; t < k; ++t) {
                    int64_t j = J[t];
                    double sign = pz[j] ? -1.0 : 1.0;
                    g[j] += w * 2.0 * sign;
                }
            }
        }
        free(J);
    }
    for (int64_t j = 0; j < m; ++j) {
        double acc = 0.0;
        for (int t = 0; t < nthreads; ++t) acc += part[(size_t)t * (size_t)m + j];
        grad[j] = acc;
    }
    free(part);
    free(PZ);
    free(PA);
}

/* Data parity sums T_a = sum_x (-1)^{a.x} over the N data rows, so that
 * <Z_a>_p = T_a / N for the empirical data distribution (Sec. 3.3.1). */
void oracle_data_parity_sum(int64_t n, const uint64_t *A, int64_t l, int64_t lda,
                            const uint64_t *X, int64_t N, int64_t ldx, int64_t *T) {
    support_t sa = support_of(A, l, lda, n);
    uint8_t *Xb = unpack_rows(X, N, ldx, n);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < l; ++a) {
        int64_t t = 0;
        for (int64_t x = 0; x < N; ++x) {
            int par = 0;
            for (int64_t k = sa.start[a]; k < sa.start[a + 1]; ++k) par ^= Xb[x * n + sa.idx[k]];
            t += par ? -1 : 1;
        }
        T[a] = t;
    }
    free(Xb);
    support_free(&sa);
}

/* MMD^2 estimate of eq. mmd_estimate over the l sampled observables, with the
 * model expectation values from the estimator (S1, S2 over the s samples)
 * and the data ones from T_a. Unbiased form (default): every square is a
 * U-statistic, i.e. the mean over ordered pairs of distinct samples,
 *   U_q = (S1^2 - S2) / (s(s-1)),  U_p = (T^2 - N) / (N(N-1)),
 * term_a = U_p - 2 (T/N)(S1/s) + U_q. Biased form: term_a = (T/N - S1/s)^2.
 * loss = (1/l) sum_a term_a. terms (l) and grad (m) may be NULL. The
 * gradient uses alpha/beta of oracle_expval_grad, from differentiating the
 * chosen form in S1 and S2. */
void oracle_expval_indep(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                         const uint64_t *A, int64_t l, int64_t lda,
                         const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                         double *expval, double *std_err, double *S1, double *S2);
void oracle_expval_indep_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                              const uint64_t *A, int64_t l, int64_t lda,
                              const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                              const double *alpha, const double *beta, double *grad);

/* Terms, loss and gradient coefficients from the per-observable sums S1, S2
 * (model) and T (data), in the form chosen by `unbiased`. */
static void mmd_terms(int64_t l, int64_t s, int64_t N, const double *S1, const double *S2, const int64_t *T,
                      int unbiased, double *loss, double *terms, double *alpha, double *beta) {
    double ds = (double)s, dN = (double)N, dl = (double)l;
    double acc = 0.0;
    for (int64_t a = 0; a < l; ++a) {
        double Td = (double)T[a];
        double p = Td / dN, q = S1[a] / ds, term;
        if (unbiased) {
            double Up = (Td * Td - dN) / (dN * (dN - 1.0));
            double Uq = (S1[a] * S1[a] - S2[a]) / (ds * (ds - 1.0));
            term = Up - 2.0 * p * q + Uq;
            /* d term / dS1 = -2p/s + 2 S1/(s(s-1)),  d term / dS2 = -1/(s(s-1));
             * dS1 = sum -sin dPhi, dS2 = sum -2 cos sin dPhi. */
            alpha[a] = (2.0 * p / ds - 2.0 * S1[a] / (ds * (ds - 1.0))) / dl;
            beta[a] = 2.0 / (ds * (ds - 1.0)) / dl;
        } else {
            term = (p - q) * (p - q);
            /* d term / dS1 = -2 (p - q) / s */
            alpha[a] = 2.0 * (p - q) / ds / dl;
            beta[a] = 0.0;
        }
        if (terms) terms[a] = term;
        acc += term;
    }
    *loss = acc / dl;
}

/* flags: 1 = unbiased form, 2 = sqrt_loss, 4 = independent batches (Z has
 * l * s rows, observable a uses rows [a s, (a+1) s)). */
void oracle_mmd_loss_ex(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                        const uint64_t *A, int64_t l, int64_t lda,
                        const uint64_t *Z, int64_t s, int64_t ldz,
                        const uint64_t *X, int64_t N, int64_t ldx, const double *theta,
                        int flags, double *loss, double *terms, double *grad) {
    const size_t L = (size_t)(l > 0 ? l : 1);
    double *S1 = (double *)malloc(sizeof(double) * L);
    double *S2 = (double *)malloc(sizeof(double) * L);
    int64_t *T = (int64_t *)malloc(sizeof(int64_t) * L);
    double *alpha = (double *)malloc(sizeof(double) * L);
    double *beta = (double *)malloc(sizeof(double) * L);
    const int indep = (flags & 4) != 0;
    if (indep)
        oracle_expval_indep(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, NULL, NULL, S1, S2);
    else
        oracle_expval(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, NULL, NULL, S1, S2);
    oracle_data_parity_sum(n, A, l, lda, X, N, ldx, T);
    mmd_terms(l, s, N, S1, S2, T, flags & 1, loss, terms, alpha, beta);
    if (grad) {
        if (indep)
            oracle_expval_indep_grad(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, alpha, beta, grad);
        else
            oracle_expval_grad(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, alpha, beta, grad);
    }
    if (flags & 2) {
        /* sqrt_loss (Sec. 3.3.1): L' = sqrt(L), dL' = dL / (2 L'); an estimate
         * L <= 0 (the unbiased form can be negative) gives L' = 0 and a zero
         * gradient. */
        double Lv = *loss;
        double r = Lv > 0.0 ? sqrt(Lv) : 0.0;
        if (grad)
            for (int64_t j = 0; j < m; ++j) grad[j] = Lv > 0.0 ? grad[j] / (2.0 * r) : 0.0;
        *loss = r;
    }
    free(beta);
    free(alpha);
    free(T);
    free(S2);
    free(S1);
}

void oracle_mmd_loss(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                     const uint64_t *A, int64_t l, int64_t lda,
                     const uint64_t *Z, int64_t s, int64_t ldz,
                     const uint64_t *X, int64_t N, int64_t ldx, const double *theta,
                     int unbiased, double *loss, double *terms, double *grad) {
    oracle_mmd_loss_ex(n, G, m, ldg, A, l, lda, Z, s, ldz, X, N, ldx, theta, unbiased ? 1 : 0, loss, terms, grad);
}

/* ---------------------------------------------------------------- exact forms */

/* Exact <Z_a> by enumerating every z in {0,1}^n (eq. op_expval with the
 * expectation taken over all 2^n strings). n <= 24. */
void oracle_exact_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                         const uint64_t *A, int64_t l, int64_t lda, const double *theta,
                         double *out) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    support_t sg = support_of(G, m, ldg, n);
    int64_t nz = (int64_t)1 << n;
#pragma omp parallel
    {
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(static)
        for (int64_t a = 0; a < l; ++a) {
            int64_t k = gates_of(PA + a * m, m, J);
            double sum = 0.0;
            for (int64_t z = 0; z < nz; ++z) {
                double phi = 0.0;
                for (int64_t t = 0; t < k; ++t) {
                    int64_t j = J[t];
                    int par = 0;
                    for (int64_t e = sg.start[j]; e < sg.start[j + 1]; ++e) par ^= (int)((z >> sg.idx[e]) & 1);
                    phi += theta[j] * (par ? -1.0 : 1.0) * 2.0;
                }
                sum += cos(phi);
            }
            out[a] = sum / (double)nz;
        }
        free(J);
    }
    support_free(&sg);
    free(PA);
}

/* Statevector of U(theta)|0> = prod_j exp(i theta_j X_{g_j}) |0> using the
 * gate action exp(i t X_g)|x> = cos t |x> + i sin t |x xor g>  (Sec. 2.5).
 * re, im have 2^n entries. n <= 26, generators on qubits < n. */
static void statevector(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const double *theta,
                        double *re, double *im) {
    int64_t dim = (int64_t)1 << n;
    double *nr = (double *)malloc(sizeof(double) * (size_t)dim);
    double *ni = (double *)malloc(sizeof(double) * (size_t)dim);
    for (int64_t x = 0; x < dim; ++x) re[x] = im[x] = 0.0;
    re[0] = 1.0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t g = 0;
        for (int64_t q = 0; q < n; ++q)
            if (bit_at(G + j * ldg, q)) g |= (int64_t)1 << q;
        double c = cos(theta[j]), sn = sin(theta[j]);
        for (int64_t x = 0; x < dim; ++x) {
            int64_t y = x ^ g;
            /* (i sn) * (re[y] + i im[y]) = -sn*im[y] + i sn*re[y] */
            nr[x] = c * re[x] - sn * im[y];
            ni[x] = c * im[x] + sn * re[y];
        }
        memcpy(re, nr, sizeof(double) * (size_t)dim);
        memcpy(im, ni, sizeof(double) * (size_t)dim);
    }
    free(ni);
    free(nr);
}

/* Output distribution q(x) = |<x|U(theta)|0>|^2 (Sec. 3.3). */
void oracle_statevector_probs(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                              const double *theta, double *probs) {
    int64_t dim = (int64_t)1 << n;
    double *re = (double *)malloc(sizeof(double) * (size_t)dim);
    double *im = (double *)malloc(sizeof(double) * (size_t)dim);
    statevector(n, G, m, ldg, theta, re, im);
    for (int64_t x = 0; x < dim; ++x) probs[x] = re[x] * re[x] + im[x] * im[x];
    free(im);
    free(re);
}

/* <Z_a> = sum_x |psi_x|^2 (-1)^{a.x}  (eq. expvals evaluated on the state). */
void oracle_statevector_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                               const uint64_t *A, int64_t l, int64_t lda, const double *theta,
                               double *out) {
    int64_t dim = (int64_t)1 << n;
    double *pr = (double *)malloc(sizeof(double) * (size_t)dim);
    oracle_statevector_probs(n, G, m, ldg, theta, pr);
    support_t sa = support_of(A, l, lda, n);
    for (int64_t a = 0; a < l; ++a) {
        double acc = 0.0;
        for (int64_t x = 0; x < dim; ++x) {
            int par = 0;
            for (int64_t e = sa.start[a]; e < sa.start[a + 1]; ++e) par ^= (int)((x >> sa.idx[e]) & 1);
            acc += par ? -pr[x] : pr[x];
        }
        out[a] = acc;
    }
    support_free(&sa);
    free(pr);
}

/* Expansion of eq. expval_intefere: with J_a the gates anticommuting with
 * Z_a, <Z_a> = sum over subsets w of J_a whose generators XOR to zero of
 *   prod_{j in J_a \ w} cos(2 theta_j) * prod_{j in w} (i sin(-2 theta_j)).
 * The empty subset gives the product term. Brute force over all 2^|J_a|
 * subsets (|J_a| <= 24), generators on qubits < 64. Such a subset has even
 * size (each of its generators has odd overlap with a), so (-i)^|w| is the
 * real (-1)^{|w|/2}. */
void oracle_subset_expansion(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                             const uint64_t *A, int64_t l, int64_t lda, const double *theta,
                             double *out) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t a = 0; a < l; ++a) {
        int64_t k = gates_of(PA + a * m, m, J);
        double acc = 0.0;
        for (int64_t w = 0; w < ((int64_t)1 << k); ++w) {
            uint64_t v = 0;
            int size = 0;
            for (int64_t t = 0; t < k; ++t)
                if ((w >> t) & 1) {
                    for (int64_t q = 0; q < n; ++q)
                        if (bit_at(G + J[t] * ldg, q)) v ^= (uint64_t)1 << q;
                    ++size;
                }
            if (v != 0) continue;
            double term = (size / 2) % 2 ? -1.0 : 1.0;
            for (int64_t t = 0; t < k; ++t) {
                double x = 2.0 * theta[J[t]];
                term *= ((w >> t) & 1) ? sin(x) : cos(x);
            }
            acc += term;
        }
        out[a] = acc;
    }
    free(J);
    free(PA);
}

/* Stochastic bitflip circuit (eq. expval_bitflip): <Z_a> = prod over J_a of
 * cos(2 theta_j). Exact for IQP circuits whose J_a has no nonempty subset
 * XORing to zero. */
void oracle_bitflip_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                           const uint64_t *A, int64_t l, int64_t lda, const double *theta,
                           double *out) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    for (int64_t a = 0; a < l; ++a) {
        double p = 1.0;
        for (int64_t j = 0; j < m; ++j)
            if (PA[a * m + j]) p *= cos(2.0 * theta[j]);
        out[a] = p;
    }
    free(PA);
}

/* Gradient of L = sum_a w_a <Z_a> for the bitflip model, by the product
 * rule on eq. expval_bitflip: d/dtheta_j prod_{k in J_a} cos(2 theta_k) =
 * -2 sin(2 theta_j) prod_{k in J_a, k != j} cos(2 theta_k) for j in J_a. */
void oracle_bitflip_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                         const uint64_t *A, int64_t l, int64_t lda, const double *theta,
                         const double *w, double *grad) {
    uint8_t *PA = parity_matrix(n, A, l, lda, G, m, ldg);
    int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) grad[j] = 0.0;
    for (int64_t a = 0; a < l; ++a) {
        int64_t k = gates_of(PA + a * m, m, J);
        for (int64_t t = 0; t < k; ++t) {
            double rest = 1.0;
            for (int64_t u = 0; u < k; ++u)
                if (u != t) rest *= cos(2.0 * theta[J[u]]);
            grad[J[t]] += w[a] * (-2.0 * sin(2.0 * theta[J[t]])) * rest;
        }
    }
    free(J);
    free(PA);
}

/* ------------------------------------------------------- API variants */

/* sqrt_loss option of the MMD loss (Sec. 3.3.1); see oracle_mmd_loss_ex. */
void oracle_mmd_loss_sqrt(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                          const uint64_t *A, int64_t l, int64_t lda,
                          const uint64_t *Z, int64_t s, int64_t ldz,
                          const uint64_t *X, int64_t N, int64_t ldx, const double *theta,
                          int unbiased, double *loss, double *grad) {
    oracle_mmd_loss_ex(n, G, m, ldg, A, l, lda, Z, s, ldz, X, N, ldx, theta, (unbiased ? 1 : 0) | 2, loss, NULL,
                       grad);
}

/* Shared-parameter gates (Sec. 3.1.1): gate p is the product of the
 * commuting exponentials of its generators, all with parameter theta_p.
 * Generators are stored gate by gate: gate p owns rows [start[p], start[p+1])
 * of G. The per-generator parameter vector is theta_gen[j] = theta_p for j in
 * gate p, and the gradient of a gate is the sum of its generators'
 * gradients (chain rule through the shared parameter). */
void oracle_expand_params(const double *theta_p, const int64_t *start, int64_t np, double *theta_gen) {
    for (int64_t p = 0; p < np; ++p)
        for (int64_t j = start[p]; j < start[p + 1]; ++j) theta_gen[j] = theta_p[p];
}

void oracle_reduce_params(const double *grad_gen, const int64_t *start, int64_t np, double *grad_p) {
    for (int64_t p = 0; p < np; ++p) {
        double acc = 0.0;
        for (int64_t j = start[p]; j < start[p + 1]; ++j) acc += grad_gen[j];
        grad_p[p] = acc;
    }
}

/* `wires` option of the MMD loss (Sec. 3.3.1): observables and data live on
 * the listed qubits only, the others are ancillas. Bit k of each source row
 * (k < nw) becomes bit wires[k] of the n-qubit destination row; every other
 * destination bit is zero. */
void oracle_embed_bits(const uint64_t *src, int64_t rows, int64_t ld_src, const int64_t *wires, int64_t nw,
                       uint64_t *dst, int64_t ld_dst) {
    for (int64_t r = 0; r < rows; ++r) {
        uint64_t *d = dst + r * ld_dst;
        for (int64_t w = 0; w < ld_dst; ++w) d[w] = 0;
        for (int64_t k = 0; k < nw; ++k)
            if (bit_at(src + r * ld_src, k)) d[wires[k] >> 6] |= (uint64_t)1 << (wires[k] & 63);
    }
}

/* indep_estimates option (Sec. 2.2, Sec. 3.1.2): observable a uses its own
 * sample batch, rows [a s, (a+1) s) of Z, so the estimates of different
 * observables are independent. Each observable is the estimator of
 * eq. expvalsample on its own batch. */
void oracle_expval_indep(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                         const uint64_t *A, int64_t l, int64_t lda,
                         const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                         double *expval, double *std_err, double *S1, double *S2) {
    for (int64_t a = 0; a < l; ++a)
        oracle_expval(n, G, m, ldg, A + a * lda, 1, lda, Z + a * s * ldz, s, ldz, theta,
                      expval ? expval + a : NULL, std_err ? std_err + a : NULL, S1 ? S1 + a : NULL,
                      S2 ? S2 + a : NULL);
}

/* Gradient of the independent-batch estimator: the sum over observables of
 * oracle_expval_grad on each observable's own batch. */
void oracle_expval_indep_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                              const uint64_t *A, int64_t l, int64_t lda,
                              const uint64_t *Z, int64_t s, int64_t ldz, const double *theta,
                              const double *alpha, const double *beta, double *grad) {
    double *g = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) grad[j] = 0.0;
    for (int64_t a = 0; a < l; ++a) {
        oracle_expval_grad(n, G, m, ldg, A + a * lda, 1, lda, Z + a * s * ldz, s, ldz, theta,
                           alpha ? alpha + a : NULL, beta ? beta + a : NULL, g);
        for (int64_t j = 0; j < m; ++j) grad[j] += g[j];
    }
    free(g);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
