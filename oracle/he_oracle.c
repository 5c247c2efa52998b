/*
 * he_oracle.c -- TEST INFRASTRUCTURE, not the product.
 *
 * A plain, slow, obviously correct CPU implementation of the CKKS evaluation
 * hot path of "Accelerating Encrypted Computing on Intel GPUs" (arXiv
 * 2109.14704). Only tests/, __graft_entry__.smoke() and the cpu_baseline leg
 * of bench.py may load it. It shares no code with the CUDA library: every
 * modular operation here is the definition, a 128-bit product reduced with
 * the C `%` operator; there is no Shoup or Barrett arithmetic, no lazy range,
 * no fused step.
 *
 * Contents and the passage each follows:
 *   or_is_prime, or_find_primes -- RNS primes below 2^60 with q = 1 mod 2N
 *                                  (Sec. II-B, RNS; Sec. III-A-1, "less than
 *                                  60 bits").
 *   or_find_psi                 -- psi, a primitive 2N-th root of unity
 *                                  (Sec. II-B); the smallest one is taken.
 *   or_ntt_fwd / or_ntt_inv     -- negacyclic NTT over Z_q[X]/(X^N+1)
 *                                  (Sec. II-B): out[i] = sum_j a_j
 *                                  psi^((2 brv(i) + 1) j), outputs in
 *                                  bit-reversed evaluation order; the inverse
 *                                  includes the factor N^-1.
 *   or_dyadic                   -- elementwise product in the NTT domain
 *                                  (Sec. II-B, the circled-dot product).
 *   or_tensor                   -- Mul (Sec. II-A): (a0b0, a0b1 + a1b0, a1b1).
 *   or_relin                    -- Relin (Sec. II-A): c' = (c0, c1) +
 *                                  round(P^-1 c[2] evk) mod q_l, RNS digits
 *                                  with one special prime P.
 *   or_rescale                  -- RS (Sec. II-A): c' = round(c / q_l) mod
 *                                  q_{l-1}.
 *
 * Pinned by tests/test_oracle_*.py against brute force (O(N^2) transforms and
 * convolutions, big-integer CRT relinearization and rescale), library
 * routines (sympy primality and n-th roots) and closed forms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

/* ---- modular arithmetic by definition ---------------------------------- */

static u64 mod_mul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 mod_add(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 mod_sub(u64 a, u64 b, u64 q) { return (u64)(((u128)(a % q) + q - (b % q)) % q); }

static u64 mod_pow(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mod_mul(r, a, q);
        a = mod_mul(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse by Fermat's little theorem (q prime) */
static u64 mod_inv(u64 a, u64 q) { return mod_pow(a, q - 2, q); }

/* ---- primes ------------------------------------------------------------ */

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every
 * n < 3.18e23 (Sorenson and Webster 2015), which covers all 64-bit n. */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = mod_pow(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = mod_mul(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* The `count` largest primes q with exactly `bits` bits and q = 1 mod two_n,
 * skipping any listed in `exclude`, in descending order. Returns the number
 * found (fewer than count only if the bit range runs out). */
int or_find_primes(int bits, u64 two_n, int count, const u64 *exclude, int n_exclude, u64 *out)
{
    if (bits < 2 || bits > 62 || two_n == 0) return 0;
    u64 hi = ((u64)1 << bits) - 1;
    u64 lo = (u64)1 << (bits - 1);
    u64 q = ((hi - 1) / two_n) * two_n + 1;
    int found = 0;
    while (found < count && q >= lo && q > two_n) {
        int skip = 0;
        for (int i = 0; i < n_exclude; i++)
            if (exclude[i] == q) skip = 1;
        if (!skip && or_is_prime(q)) out[found++] = q;
        q -= two_n;
    }
    return found;
}

/* ---- psi, the primitive 2N-th root -------------------------------------- */

/* The smallest psi in [2, q) with psi^N = -1 mod q (for N a power of two that
 * is exactly a primitive 2N-th root). Every primitive 2N-th root is an odd
 * power of any one of them, g^((q-1)/2N) for a quadratic non-residue g. */
u64 or_find_psi(u64 q, u64 N)
{
    if (N == 0 || (q - 1) % (2 * N) != 0) return 0;
    u64 g = 2;
    while (mod_pow(g, (q - 1) / 2, q) != q - 1) g++;
    u64 root = mod_pow(g, (q - 1) / (2 * N), q);
    u64 sq = mod_mul(root, root, q);
    u64 best = root, x = root;
    for (u64 k = 1; k < N; k++) {
        x = mod_mul(x, sq, q);
        if (x < best) best = x;
    }
    return best;
}

static u64 bit_reverse(u64 x, int logn)
{
    u64 r = 0;
    for (int i = 0; i < logn; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

static int log2_exact(u64 n)
{
    int l = 0;
    while (((u64)1 << l) < n) l++;
    return l;
}

/* ---- negacyclic NTT (Sec. II-B) ---------------------------------------- */

/* Forward transform in place. With the psi-twist folded into the twiddles,
 * the radix-2 Cooley-Tukey network over bit-reversed powers of psi computes
 * out[i] = sum_j a_j psi^((2 brv(i) + 1) j) (Longa and Naehrig 2016, cited in
 * Sec. II-B). Stage m (m = 1, 2, ..., N/2) has m groups; group i uses
 * W = psi^brv(m + i) and pairs positions j and j + N/(2m). */
void or_ntt_fwd(u64 *a, u64 N, u64 q, u64 psi)
{
    int logn = log2_exact(N);
    u64 *tw = (u64 *)malloc(N * sizeof(u64));
    for (u64 k = 0; k < N; k++) tw[k] = mod_pow(psi, bit_reverse(k, logn), q);
    u64 t = N;
    for (u64 m = 1; m < N; m *= 2) {
        t /= 2;
        for (u64 i = 0; i < m; i++) {
            u64 w = tw[m + i];
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 x = a[j], y = mod_mul(w, a[j + t], q);
                a[j] = mod_add(x, y, q);
                a[j + t] = mod_sub(x, y, q);
            }
        }
    }
    free(tw);
}

/* Inverse transform in place: undoes the forward stages in reverse order. The
 * inverse of (x, y) -> (x + W y, x - W y) is (x, y) -> ((x + y)/2,
 * (x - y) W^-1 / 2); the factors 1/2 of all log N stages give the N^-1
 * applied at the end. */
void or_ntt_inv(u64 *a, u64 N, u64 q, u64 psi)
{
    int logn = log2_exact(N);
    u64 psi_inv = mod_inv(psi, q);
    u64 *tw = (u64 *)malloc(N * sizeof(u64));
    for (u64 k = 0; k < N; k++) tw[k] = mod_pow(psi_inv, bit_reverse(k, logn), q);
    u64 t = 1;
    for (u64 m = N / 2; m >= 1; m /= 2) {
        for (u64 i = 0; i < m; i++) {
            u64 w = tw[m + i];
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 x = a[j], y = a[j + t];
                a[j] = mod_add(x, y, q);
                a[j + t] = mod_mul(mod_sub(x, y, q), w, q);
            }
        }
        t *= 2;
    }
    u64 n_inv = mod_inv(N % q, q);
    for (u64 j = 0; j < N; j++) a[j] = mod_mul(a[j], n_inv, q);
    free(tw);
}

/* ---- NTT-domain products (Sec. II-A Mul, Sec. II-B) -------------------- */

void or_dyadic(u64 *out, const u64 *a, const u64 *b, u64 N, u64 q)
{
    for (u64 i = 0; i < N; i++) out[i] = mod_mul(a[i], b[i], q);
}

/* Mul: ciphertexts are [component][limb][N] in the NTT domain, n limbs.
 * out = (a0 b0, a0 b1 + a1 b0, a1 b1), 3 components. */
void or_tensor(u64 *out, const u64 *ca, const u64 *cb, u64 N, int n, const u64 *moduli)
{
    u64 comp = (u64)n * N;
    for (int l = 0; l < n; l++) {
        u64 q = moduli[l];
        const u64 *a0 = ca + l * N, *a1 = ca + comp + l * N;
        const u64 *b0 = cb + l * N, *b1 = cb + comp + l * N;
        u64 *d0 = out + l * N, *d1 = out + comp + l * N, *d2 = out + 2 * comp + l * N;
        for (u64 i = 0; i < N; i++) {
            d0[i] = mod_mul(a0[i], b0[i], q);
            d1[i] = mod_add(mod_mul(a0[i], b1[i], q), mod_mul(a1[i], b0[i], q), q);
            d2[i] = mod_mul(a1[i], b1[i], q);
        }
    }
}

/* ---- Relin (Sec. II-A) ------------------------------------------------- */

/* c' = (c0, c1) + round(P^-1 * c[2] * evk) mod q_l, with c[2] decomposed into
 * its RNS digits c2_j = [c[2]]_{q_j} in [0, q_j), j = 0..l, and one special
 * prime P. Key layout: evk[j][k][t][N], j < n_max digits, k in {0, 1}, t over
 * the n_max data limbs followed by P (n_max + 1 limbs), NTT domain. At level l
 * the digits 0..l and the limbs {q_0..q_l, P} are used.
 *
 * Steps: (i) c2_j = INTT_{q_j}(d2[j]); (ii) for every target modulus t in
 * {q_0..q_l, P}: acc_k[t] = sum_j NTT_t(c2_j mod t) * evk[j][k][t];
 * (iii) division by P with rounding: y = INTT_P(acc_k[P]), r = the centred
 * residue of y mod P (in [-(P-1)/2, (P-1)/2]), and for each q_i
 * out_k[i] = (acc_k[q_i] - NTT_{q_i}(r mod q_i)) * P^-1; (iv) c'_k = d_k +
 * out_k. ct_in is [3][n][N], ct_out is [2][n][N], n = level + 1. */
void or_relin(u64 *ct_out, const u64 *ct_in, const u64 *evk, u64 N, int n_max,
              const u64 *moduli, u64 P, int level)
{
    int n = level + 1;
    u64 comp = (u64)n * N;
    int nt = n + 1; /* targets q_0..q_l, P */
    u64 *tmod = (u64 *)malloc(nt * sizeof(u64));
    u64 *tpsi = (u64 *)malloc(nt * sizeof(u64));
    for (int t = 0; t < n; t++) tmod[t] = moduli[t];
    tmod[n] = P;
    for (int t = 0; t < nt; t++) tpsi[t] = or_find_psi(tmod[t], N);

    /* (i) digits in the coefficient domain */
    u64 *c2 = (u64 *)malloc(comp * sizeof(u64));
    memcpy(c2, ct_in + 2 * comp, comp * sizeof(u64));
    for (int j = 0; j < n; j++) or_ntt_inv(c2 + (u64)j * N, N, tmod[j], tpsi[j]);

    /* (ii) accumulate digit x key products for every target modulus */
    u64 *acc = (u64 *)calloc((u64)2 * nt * N, sizeof(u64)); /* [k][t][N] */
    u64 *r = (u64 *)malloc(N * sizeof(u64));
    for (int t = 0; t < nt; t++) {
        u64 q = tmod[t];
        int key_limb = (t < n) ? t : n_max; /* P sits after the n_max data limbs */
        for (int j = 0; j < n; j++) {
            for (u64 i = 0; i < N; i++) r[i] = c2[(u64)j * N + i] % q;
            or_ntt_fwd(r, N, q, tpsi[t]);
            for (int k = 0; k < 2; k++) {
                const u64 *key = evk + (((u64)j * 2 + k) * (n_max + 1) + key_limb) * N;
                u64 *a = acc + ((u64)k * nt + t) * N;
                for (u64 i = 0; i < N; i++) a[i] = mod_add(a[i], mod_mul(r[i], key[i], q), q);
            }
        }
    }

    /* (iii) divide by P with rounding, (iv) add (c0, c1) */
    u64 half = (P - 1) / 2;
    u64 *y = (u64 *)malloc(N * sizeof(u64));
    for (int k = 0; k < 2; k++) {
        memcpy(y, acc + ((u64)k * nt + n) * N, N * sizeof(u64));
        or_ntt_inv(y, N, P, tpsi[n]);
        for (int t = 0; t < n; t++) {
            u64 q = tmod[t];
            u64 p_inv = mod_inv(P % q, q);
            for (u64 i = 0; i < N; i++) {
                /* centred residue: y - P if y > (P-1)/2, as an integer mod q */
                r[i] = (y[i] <= half) ? y[i] % q : mod_sub(y[i] % q, P % q, q);
            }
            or_ntt_fwd(r, N, q, tpsi[t]);
            const u64 *a = acc + ((u64)k * nt + t) * N;
            const u64 *d = ct_in + (u64)k * comp + (u64)t * N;
            u64 *o = ct_out + (u64)k * comp + (u64)t * N;
            for (u64 i = 0; i < N; i++)
                o[i] = mod_add(d[i], mod_mul(mod_sub(a[i], r[i], q), p_inv, q), q);
        }
    }
    free(y); free(r); free(acc); free(c2); free(tpsi); free(tmod);
}

/* ---- RS (Sec. II-A) ---------------------------------------------------- */

/* c' = round(c / q_l) mod Q_{l-1} for both components. The last limb is
 * brought to the coefficient domain, its centred residue r (in
 * [-(q_l-1)/2, (q_l-1)/2]) is subtracted so that c - r is divisible by q_l,
 * and each remaining limb becomes (c_i - NTT_{q_i}(r mod q_i)) * q_l^-1.
 * ct_in is [2][l+1][N], ct_out is [2][l][N], level l >= 1. */
void or_rescale(u64 *ct_out, const u64 *ct_in, u64 N, const u64 *moduli, int level)
{
    int n = level + 1;
    u64 ql = moduli[level];
    u64 half = (ql - 1) / 2;
    u64 psi_l = or_find_psi(ql, N);
    u64 *y = (u64 *)malloc(N * sizeof(u64));
    u64 *r = (u64 *)malloc(N * sizeof(u64));
    for (int k = 0; k < 2; k++) {
        memcpy(y, ct_in + ((u64)k * n + level) * N, N * sizeof(u64));
        or_ntt_inv(y, N, ql, psi_l);
        for (int t = 0; t < level; t++) {
            u64 q = moduli[t];
            u64 inv = mod_inv(ql % q, q);
            for (u64 i = 0; i < N; i++)
                r[i] = (y[i] <= half) ? y[i] % q : mod_sub(y[i] % q, ql % q, q);
            or_ntt_fwd(r, N, q, or_find_psi(q, N));
            const u64 *c = ct_in + ((u64)k * n + t) * N;
            u64 *o = ct_out + ((u64)k * level + t) * N;
            for (u64 i = 0; i < N; i++) o[i] = mod_mul(mod_sub(c[i], r[i], q), inv, q);
        }
    }
    free(r); free(y);
}

/* ---- helpers for the host-side CKKS routines --------------------------- */

/* Negacyclic product c = a * b in Z_q[X]/(X^N+1) through the convolution
 * theorem of Sec. II-B: INTT(NTT(a) . NTT(b)). */
void or_negacyclic_mul(u64 *c, const u64 *a, const u64 *b, u64 N, u64 q, u64 psi)
{
    u64 *ta = (u64 *)malloc(N * sizeof(u64));
    memcpy(ta, a, N * sizeof(u64));
    memcpy(c, b, N * sizeof(u64));
    or_ntt_fwd(ta, N, q, psi);
    or_ntt_fwd(c, N, q, psi);
    or_dyadic(c, ta, c, N, q);
    or_ntt_inv(c, N, q, psi);
    free(ta);
}

u64 or_pow_mod(u64 a, u64 e, u64 q) { return mod_pow(a, e, q); }
u64 or_mul_mod(u64 a, u64 b, u64 q) { return mod_mul(a, b, q); }
