/*
 * Oracle for the MoA ONF GEMM -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct CPU statement of what the
 * product path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library and includes nothing from it.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -fPIC -shared
 * (no fused multiply-add: every product is rounded, then added).
 *
 * Contents
 *   moa_oracle_gemm_f64        Eq. (eq:dnf), Sec. 2: C[(i*p)+j] := sum_k A[(i*n)+k]*B[(k*p)+j]
 *   moa_oracle_gemm_f64_rows   the same, for a chosen subset of rows i
 *   moa_oracle_gemm_f64_omp    the same, rows dealt to threads (the ip_rows lift, Sec. 3.1)
 *   moa_oracle_split3_bf16     precision slicing, FP32-accuracy mode (not in the paper)
 *   moa_oracle_slice_fixed     precision slicing, FP64-accuracy mode (not in the paper)
 *   moa_oracle_split_gemm_exact  the value the FP64-accuracy slice method reaches
 *   moa_oracle_crt_moduli      moduli of the FP64-accuracy modular-slice mode (not in the paper)
 *   moa_oracle_crt_bits        operand bits that mode keeps for a given n and modulus count
 *   moa_oracle_scale_int       per-row / per-column scaling of an operand to integers
 *   moa_oracle_int_gemm_exact  the value the modular-slice method reaches
 *   moa_oracle_kronecker_f64   Kronecker product (Appendix: outer product, no reduction)
 *   moa_oracle_hadamard_f64    Hadamard product (Appendix: diagonal of the outer product)
 *
 * Parity status: the GEMM functions are pinned by exact-integer, identity,
 * permutation, transpose, associativity and exact-rational (Higham bound)
 * tests.  The slicing functions are pinned by exact reconstruction, range and
 * library-rounding tests.  moa_oracle_split_gemm_exact is pinned against the
 * GEMM oracle within the slicing error bound.  The Kronecker and Hadamard
 * products are pinned by the mixed-product property, identities and the
 * trace identity on integer inputs.  The modular-slice functions are pinned
 * by coprimality and maximality of the moduli, the bit bound checked with
 * big integers, an exact-rational route for the scaling, and brute force,
 * exact-integer and truncation-bound tests of the exact product.
 */
#include <stdint.h>
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One row i of Eq. (eq:dnf) in the order of Fig. ip.c: the row of C is
 * cleared (the equation assigns, the figure accumulates into a zeroed C),
 * then for k = 0..n-1 the scalar A[i,k] scales the contiguous row k of B and
 * is added into the contiguous row i of C (Fig. fig:mm). */
static void onf_row(int64_t i, int64_t n, int64_t p,
                    const double* A, const double* B, double* Crow)
{
    for (int64_t j = 0; j < p; ++j) Crow[j] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double a = A[i * n + k];
        const double* Brow = B + k * p;
        for (int64_t j = 0; j < p; ++j) {
            const double prod = a * Brow[j];
            Crow[j] = Crow[j] + prod;
        }
    }
}

/* C (m x p) := A (m x n) . B (n x p); all row-major, FP64.  Eq. (eq:dnf). */
void moa_oracle_gemm_f64(int64_t m, int64_t n, int64_t p,
                         const double* A, const double* B, double* C)
{
    for (int64_t i = 0; i < m; ++i) onf_row(i, n, p, A, B, C + i * p);
}

/* Rows rows[0..nrows) of C, written densely into Crows (nrows x p). */
void moa_oracle_gemm_f64_rows(int64_t m, int64_t n, int64_t p,
                              const double* A, const double* B,
                              int64_t nrows, const int64_t* rows, double* Crows)
{
    (void)m;
    for (int64_t r = 0; r < nrows; ++r) onf_row(rows[r], n, p, A, B, Crows + r * p);
}

/* Rows of C dealt to `threads` OpenMP threads: the i-loop lift of Sec. 3.1
 * (Fig. ip_rows.c) with each processor owning whole rows.  Per element the
 * arithmetic is that of onf_row, so the result is bit-identical to
 * moa_oracle_gemm_f64.  Returns the number of threads actually used. */
int moa_oracle_gemm_f64_omp(int64_t m, int64_t n, int64_t p,
                            const double* A, const double* B, double* C, int threads)
{
    int used = 1;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_num_procs();
#pragma omp parallel num_threads(threads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; ++i) onf_row(i, n, p, A, B, C + i * p);
    }
#else
    (void)threads;
    moa_oracle_gemm_f64(m, n, p, A, B, C);
#endif
    return used;
}

/* ------------------------------------------------------------------------ */
/* Precision slicing, FP32-accuracy mode.  Not in the paper: the split of    */
/* Henry, Tang & Heinecke (2019).  Each FP32 value x is written as           */
/* x = s0 + s1 + s2 with s_t = RN_bf16(x - (s0 + ... + s_{t-1})).            */
/* ------------------------------------------------------------------------ */

/* Round an FP32 value to the nearest BF16 value, ties to even, returned as
 * FP32.  BF16 keeps the FP32 sign and exponent and the top 7 fraction bits,
 * so rounding is done on the bit pattern: add half of the dropped unit
 * (minus one when the kept part is even) and clear the dropped 16 bits.
 * NaN stays NaN; values that round past the largest finite BF16 become Inf,
 * as IEEE rounding prescribes. */
static float round_to_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0u) {
        u |= 0x00400000u;            /* quiet NaN, keep the payload's top bits */
        u &= 0xffff0000u;
    } else {
        const uint32_t keep_lsb = (u >> 16) & 1u;
        u += 0x7fffu + keep_lsb;
        u &= 0xffff0000u;
    }
    float r;
    memcpy(&r, &u, sizeof r);
    return r;
}

/* s0, s1, s2 (each `count` values, BF16 values stored as FP32) of x. */
void moa_oracle_split3_bf16(int64_t count, const float* x,
                            float* s0, float* s1, float* s2)
{
    for (int64_t e = 0; e < count; ++e) {
        const float v = x[e];
        const float a = round_to_bf16(v);
        const float r1 = v - a;           /* exact: a holds v's leading bits */
        const float b = round_to_bf16(r1);
        const float r2 = r1 - b;          /* exact for the same reason */
        const float c = round_to_bf16(r2);
        s0[e] = a; s1[e] = b; s2[e] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* Precision slicing, FP64-accuracy mode.  Not in the paper: error-free      */
/* slicing in the manner of Ozaki, Ogita, Oishi & Rump (2012).               */
/* Each group (a row of A, or a column of B) gets the exponent e = f + h,    */
/* where max|x| over the group lies in [2^(f-1), 2^f) (f = 0 for an          */
/* all-zero group) and h >= 0 is the headroom: bits left unused above the    */
/* top digit.  Each x of the group is scaled to X = x * 2^(beta*S - e), so   */
/* |X| < 2^(beta*S - h), and rounded once to the nearest integer D (ties to  */
/* even).  D is then written in balanced radix 2^beta with S digits:         */
/*   D = sum_{s=0}^{S-1} d_s 2^(beta(S-1-s)),                                */
/*   d_s in [-2^(beta-1), 2^(beta-1)) for s >= 1 (taken from the bottom),   */
/*   |d_0| <= 2^(beta-h),                                                    */
/* so that |x - 2^e sum_s d_s 2^(-beta(s+1))| <= 2^(e - beta S) / 2.         */
/* h = 0 suits BF16 digit planes (beta <= 8: every |d| <= 2^beta is a BF16   */
/* value); h = 1 with beta = 5 keeps every digit within [-16, 16], the       */
/* integers that FP8 E4M3 holds exactly.                                     */
/* ------------------------------------------------------------------------ */

/* X is rows x cols row-major.  axis 0: one exponent per row (length rows);
 * axis 1: one exponent per column (length cols).  digits is S x rows x cols
 * (slice-major), int32.  Requires beta * S <= 60 and 0 <= headroom < beta. */
void moa_oracle_slice_fixed(int64_t rows, int64_t cols, const double* X,
                            int axis, int beta, int S, int headroom,
                            int32_t* exps, int32_t* digits)
{
    const int64_t ngroups = axis == 0 ? rows : cols;
    for (int64_t g = 0; g < ngroups; ++g) {
        double mu = 0.0;
        const int64_t len = axis == 0 ? cols : rows;
        for (int64_t q = 0; q < len; ++q) {
            const double v = axis == 0 ? X[g * cols + q] : X[q * cols + g];
            const double av = fabs(v);
            if (av > mu) mu = av;
        }
        int f = 0;
        if (mu != 0.0) (void)frexp(mu, &f);     /* mu = q * 2^f, q in [1/2, 1) */
        exps[g] = f + headroom;
    }
    const int64_t radix = (int64_t)1 << beta;
    const int64_t half = radix / 2;
    for (int64_t r = 0; r < rows; ++r) {
        for (int64_t c = 0; c < cols; ++c) {
            const int e = axis == 0 ? exps[r] : exps[c];
            /* x * 2^(beta S - e) is exact (|X| < 2^60, no overflow; a result
             * in the subnormal range rounds to 0 below anyway), and rint in
             * the default rounding mode rounds half to even. */
            int64_t D = (int64_t)rint(ldexp(X[r * cols + c], beta * S - e));
            for (int s = S - 1; s >= 1; --s) {
                int64_t low = D % radix;               /* C remainder: sign of D */
                if (low < 0) low += radix;             /* now in [0, radix) */
                if (low >= half) low -= radix;         /* balanced: [-half, half) */
                digits[((int64_t)s * rows + r) * cols + c] = (int32_t)low;
                D = (D - low) / radix;                 /* exact division */
            }
            digits[((int64_t)0 * rows + r) * cols + c] = (int32_t)D;
        }
    }
}

/* mag * 2^exp2 rounded to the nearest FP64 value, ties to even, with a
 * single rounding (results in the subnormal range round twice). */
static double u128_scaled_to_double(unsigned __int128 mag, int exp2)
{
    if (mag == 0) return 0.0;
    const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
    const int nbits = hi ? 128 - __builtin_clzll(hi) : 64 - __builtin_clzll(lo);
    if (nbits <= 53) return ldexp((double)lo, exp2);
    const int drop = nbits - 53;
    unsigned __int128 q = mag >> drop;
    const unsigned __int128 rem = mag - (q << drop);
    const unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
    if (rem > half || (rem == half && (q & 1u))) q += 1;   /* q <= 2^53: exact */
    return ldexp((double)(uint64_t)q, exp2 + drop);
}

/* The value the FP64-accuracy slice method reaches, computed exactly and
 * rounded once:
 *   C[i,j] = 2^(eA_i + eB_j) * sum_{s+t <= S-1} 2^(-beta(s+t+2)) *
 *            sum_k dA_s[i,k] * dB_t[k,j]
 * for digits dA (per-row exponents of A) and dB (per-column exponents of B)
 * as produced by moa_oracle_slice_fixed.  The inner sums are exact in int64;
 * the levels are combined in a 128-bit integer at the finest level's scale
 * and converted to FP64 with one rounding.  Requires n * 2^(2 beta) * S < 2^62
 * (each level sum fits int64) and beta * (S - 1) + 62 < 127 (the shifted
 * level sums fit the 128-bit total). */
void moa_oracle_split_gemm_exact(int64_t m, int64_t n, int64_t p,
                                 const int32_t* dA, const int32_t* eA,
                                 const int32_t* dB, const int32_t* eB,
                                 int beta, int S, double* C)
{
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < p; ++j) {
            __int128 total = 0;                     /* units of 2^(-beta(S+1)) */
            for (int level = 0; level < S; ++level) {
                int64_t lev = 0;
                for (int s = 0; s <= level; ++s) {
                    const int t = level - s;
                    const int32_t* a = dA + ((int64_t)s * m + i) * n;
                    const int32_t* b = dB + (int64_t)t * n * p + j;
                    for (int64_t k = 0; k < n; ++k)
                        lev += (int64_t)a[k] * (int64_t)b[k * p];
                }
                total += (__int128)lev << (beta * (S - 1 - level));
            }
            /* total * 2^(-beta(S+1)) * 2^(eA+eB), rounded once. */
            const int neg = total < 0;
            const unsigned __int128 mag = neg ? (unsigned __int128)(-total)
                                              : (unsigned __int128)total;
            const double v = u128_scaled_to_double(mag, (int)(eA[i] + eB[j]) - beta * (S + 1));
            C[i * p + j] = neg ? -v : v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 accuracy from modular slices (not in the paper; the residue-number   */
/* form of error-free slicing, in the manner of Ozaki, Uchino & Imamura's   */
/* "Ozaki scheme II", 2025).  Each row i of A is scaled by 2^(t - eA_i) and rounded to an        */
/* integer A'[i,k] (|A'| <= 2^t), each column j of B by 2^(t - eB_j) to      */
/* B'[k,j]; the integer product C' = A' B' is exact, and                     */
/*     C[i,j] = C'[i,j] * 2^(eA_i + eB_j - 2t), rounded once to FP64.         */
/* A GPU forms C' from its residues modulo M pairwise-coprime moduli (one    */
/* small exact GEMM per modulus) by the Chinese remainder theorem, which     */
/* recovers C' itself when n * 2^(2t) < P / 2, P the product of the moduli.  */
/* The functions below state that definition; the residues are the GPU's    */
/* business, so none is formed here.                                         */
/* ------------------------------------------------------------------------ */

static int64_t gcd64(int64_t a, int64_t b)
{
    while (b != 0) { const int64_t r = a % b; a = b; b = r; }
    return a;
}

/* The first M integers of the sequence 256, 255, 254, ... that are coprime
 * to every integer taken before them (a greedy, descending choice; every
 * modulus is at most 2^8 so that each symmetric residue is an integer of
 * magnitude <= 128, exact in BF16).  Requires 1 <= M <= 20. */
void moa_oracle_crt_moduli(int M, int32_t* out)
{
    int taken = 0;
    for (int64_t c = 256; c >= 2 && taken < M; --c) {
        int ok = 1;
        for (int q = 0; q < taken; ++q)
            if (gcd64(c, out[q]) != 1) { ok = 0; break; }
        if (ok) out[taken++] = (int32_t)c;
    }
}

/* Largest t <= 62 with n * 2^(2t + 1) < P (P the product of the first M
 * moduli): with |A'|, |B'| <= 2^t every |C'| <= n 2^(2t) < P / 2, so the
 * symmetric residue class modulo P names C' uniquely.  Requires
 * 1 <= M <= 16 (P < 2^128) and n >= 1; returns -1 if no t >= 0 fits. */
int moa_oracle_crt_bits(int64_t n, int M)
{
    int32_t mod[16];
    moa_oracle_crt_moduli(M, mod);
    unsigned __int128 P = 1;
    for (int q = 0; q < M; ++q) P *= (unsigned __int128)mod[q];
    int best = -1;
    for (int t = 0; t <= 62; ++t) {
        /* n * 2^(2t+1) < P  <=>  n < P / 2^(2t+1) (exact: compare n with the
         * ceiling of the quotient) */
        const int sh = 2 * t + 1;
        if (sh >= 128) break;
        const unsigned __int128 q = P >> sh;
        const int exact = (q << sh) == P;
        /* n * 2^sh < P  <=>  n < P / 2^sh  <=>  n <= ceil(P / 2^sh) - 1 */
        const unsigned __int128 lim = exact ? q - 1 : q;
        if ((unsigned __int128)n <= lim) best = t;
        else break;
    }
    return best;
}

/* Per-group exponents and scaled integers of X (rows x cols, row-major):
 * axis 0 scales each row, axis 1 each column.  e_g is the frexp exponent of
 * the group's largest magnitude (0 for an all-zero group), so that every
 * |x| < 2^e_g, and ints[r,c] = x * 2^(t - e_g) rounded to the nearest
 * integer, ties to even: |ints| <= 2^t.  Requires 0 <= t <= 62. */
void moa_oracle_scale_int(int64_t rows, int64_t cols, const double* X, int axis, int t,
                          int32_t* exps, int64_t* ints)
{
    const int64_t ngroups = axis == 0 ? rows : cols;
    for (int64_t g = 0; g < ngroups; ++g) {
        double mu = 0.0;
        const int64_t len = axis == 0 ? cols : rows;
        for (int64_t q = 0; q < len; ++q) {
            const double v = axis == 0 ? X[g * cols + q] : X[q * cols + g];
            if (fabs(v) > mu) mu = fabs(v);
        }
        int f = 0;
        if (mu != 0.0) (void)frexp(mu, &f);
        exps[g] = f;
    }
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            const int e = axis == 0 ? exps[r] : exps[c];
            /* the scaling by a power of two is exact unless the result is
             * subnormal, and such a result (< 2^-1022) rounds to 0 anyway;
             * rint rounds half to even in the default rounding mode */
            ints[r * cols + c] = (int64_t)rint(ldexp(X[r * cols + c], t - e));
        }
}

/* C[i,j] = (sum_k Ai[i,k] * Bi[k,j]) * 2^(eA_i + eB_j - 2t), the sum exact in
 * 128-bit integers, rounded once to FP64.  Requires |Ai|, |Bi| <= 2^62 and
 * n * max|Ai| * max|Bi| < 2^127. */
void moa_oracle_int_gemm_exact(int64_t m, int64_t n, int64_t p,
                               const int64_t* Ai, const int32_t* eA,
                               const int64_t* Bi, const int32_t* eB,
                               int t, double* C)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < p; ++j) {
            __int128 acc = 0;
            for (int64_t k = 0; k < n; ++k)
                acc += (__int128)Ai[i * n + k] * (__int128)Bi[k * p + j];
            const int neg = acc < 0;
            const unsigned __int128 mag = neg ? (unsigned __int128)(-acc)
                                              : (unsigned __int128)acc;
            const double v = u128_scaled_to_double(mag, (int)(eA[i] + eB[j]) - 2 * t);
            C[i * p + j] = neg ? -v : v;
        }
}

/* ------------------------------------------------------------------------ */
/* The other products of the inner/outer-product family (paper's Appendix). */
/* With the outer product T[i,j,k,l] = A[i,j] * B[k,l]:                      */
/*   Kronecker  C[(i*p)+k, (j*q)+l] = T[i,j,k,l]                             */
/*   Hadamard   C[i,j] = T[i,j,i,j]                                          */
/* ------------------------------------------------------------------------ */

/* A m x n, B p x q, C (m*p) x (n*q), all row-major FP64. */
void moa_oracle_kronecker_f64(int64_t m, int64_t n, int64_t p, int64_t q,
                              const double* A, const double* B, double* C)
{
    const int64_t ncols = n * q;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t k = 0; k < p; ++k)
                for (int64_t l = 0; l < q; ++l)
                    C[(i * p + k) * ncols + (j * q + l)] = A[i * n + j] * B[k * q + l];
}

/* C[i,j] = A[i,j] * B[i,j] over m x n arrays, FP64. */
void moa_oracle_hadamard_f64(int64_t m, int64_t n, const double* A, const double* B, double* C)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            C[i * n + j] = A[i * n + j] * B[i * n + j];
}
