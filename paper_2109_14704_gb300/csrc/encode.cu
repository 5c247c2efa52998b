// encode.cu -- CKKS encoding and decoding on the device (Sec. II-A).
//
// A message is n = N/2 complex slots; slot j is the value of the real
// plaintext polynomial m at the root zeta^(5^j mod 2N), zeta = exp(i pi / N).
// Because 5^j = 4 t_j + 1 runs over every residue 1 mod 4 of 2N exactly once
// (t_j is a permutation of [0, n)) and zeta^(n (4t + 1)) = i,
//   z_j = sum_{k<n} (m_k + i m_{k+n}) zeta^k exp(2 pi i t_j k / n),
// an n-point complex DFT of the twisted vector w_k zeta^k, w_k = m_k + i m_{k+n},
// read at index t_j. Decoding is that DFT; encoding is its inverse:
// X_{t_j} = Delta z_j, u = DFT^-(X) / n, w_k = u_k zeta^-k, then m_k and
// m_{k+n} are the rounded real and imaginary parts of w_k. The DFT runs in
// FP64 as a four-step FFT (n = n1 n2): pass A, n2 transforms of length n1
// over the columns followed by the twiddles omega^(k2 t1); pass B, n1
// transforms of length n2 over the rows. Each pass is a batch of short
// radix-4 (and one radix-2) transforms in shared memory (2^10 complex values
// per CTA: more CTAs than SMs several times over, so the last wave is short).
//
// Decoding first lifts the RNS residues of every coefficient to the nearest
// double of the centred integer in (-Q/2, Q/2): a multi-word sum
// sum_i [c_i (Q/q_i)^-1]_{q_i} (Q/q_i), minus the multiple of Q that a
// floating-point estimate from the sum's top two words gives, with an exact
// multi-word correction, and a correctly rounded conversion (the mantissa is
// the top 64 bits with a sticky bit for the rest).
#include <math.h>

#include <algorithm>

#include "launch.h"

namespace he {

static const int kLogTile = 10;   // complex values per CTA of an FFT pass
static const int kFftThreads = 256;

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 c_conj_if(double2 a, bool c) { return c ? make_double2(a.x, -a.y) : a; }

// One FFT pass over a tile of G sequences of length L (G L <= 2^kLogTile)
// of message `msg`. PASS 0 is the column pass (sequence k2 < n2, element
// k1 < n1 at index k1 n2 + k2), PASS 1 the row pass (sequence t1 < n1,
// element k2 < n2 at index t1 n2 + k2 of the pass-A output). Shared memory
// holds element (g, k) at sm[k (G + 1) + g] (the padding keeps both the
// row-major loads and the column-major butterflies free of bank conflicts).
// MODE: 0 = encode (DFT with exp(-2 pi i / n)), 1 = decode (exp(+2 pi i / n)).
template <int MODE, int PASS>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(FftArgs a)
{
    extern __shared__ double2 sm[];
    const u32 n = 1u << a.log_n;
    const u32 log_L = PASS == 0 ? a.log_n1 : a.log_n - a.log_n1;
    const u32 L = 1u << log_L;
    const u32 log_seqs = a.log_n - log_L;
    const u32 log_G = min(log_seqs, (u32)kLogTile - log_L);
    const u32 G = 1u << log_G, P = G + 1;
    const u32 log_tiles = log_seqs - log_G;
    const u32 msg = blockIdx.x >> log_tiles;
    const u32 s0 = (blockIdx.x & ((1u << log_tiles) - 1)) << log_G;
    const u32 n2 = 1u << (a.log_n - a.log_n1);
    const bool conj = MODE == 1;   // decode transforms with the conjugate roots
    const u32 tile = G << log_L;

    // ---- load
    if constexpr (PASS == 0) {
        for (u32 e = threadIdx.x; e < tile; e += kFftThreads) {
            const u32 g = e & (G - 1), k = e >> log_G;
            const u32 p = (k << (a.log_n - a.log_n1)) + s0 + g;   // FFT input index
            double2 x;
            if constexpr (MODE == 0) {
                const double2 z = a.z_in[(size_t)msg * n + a.slot_of[p]];
                x = make_double2(z.x * a.scale, z.y * a.scale);
            } else {
                const double *m = a.m_in + (size_t)msg * 2 * n;
                x = c_mul(make_double2(m[p], m[p + n]), a.zeta[p]);
            }
            sm[k * P + g] = x;
        }
    } else {
        for (u32 e = threadIdx.x; e < tile; e += kFftThreads) {
            const u32 k = e & (L - 1), g = e >> log_L;
            sm[k * P + g] = a.u[(size_t)msg * n + (size_t)(s0 + g) * n2 + k];
        }
    }
    __syncthreads();

    // ---- decimation in frequency: natural order in, bit-reversed out. Groups
    // of 2^log_g elements; an odd number of stages starts with one radix-2
    // stage, the rest are radix-4 stages (two radix-2 stages with 3 twiddle
    // products instead of 4): for a quarter span h and j < h,
    //   a = x0 + x2, b = x1 + x3, c = x0 - x2, d = (x1 - x3) W_4,
    //   (x0, x1, x2, x3) <- (a + b, (a - b) W^2j, (c + d) W^j, (c - d) W^3j),
    // W = W_{4h} = omega^(n / 4h) and W_4 = -i (its conjugates for decoding).
    u32 log_g = log_L;
    if (log_L & 1) {
        const u32 lh = log_L - 1, h = 1u << lh;
        for (u32 b = threadIdx.x; b < tile / 2; b += kFftThreads) {
            const u32 g = b & (G - 1), j = b >> log_G;
            const u32 r = j & (h - 1), k = ((j >> lh) << (lh + 1)) | r;
            double2 *px = sm + k * P + g, *py = px + h * P;
            const double2 x = *px, y = *py;
            const double2 w = c_conj_if(a.omega[r << (a.log_n - lh - 1)], conj);   // W_{2h}^r
            *px = c_add(x, y);
            *py = c_mul(c_sub(x, y), w);
        }
        __syncthreads();
        log_g = lh;
    }
    for (; log_g >= 2; log_g -= 2) {
        const u32 lq = log_g - 2, h = 1u << lq, hp = h * P, sh = a.log_n - log_g;
        for (u32 b = threadIdx.x; b < tile / 4; b += kFftThreads) {
            const u32 g = b & (G - 1), j = b >> log_G;
            const u32 r = j & (h - 1), k = ((j >> lq) << (lq + 2)) | r;
            double2 *p0 = sm + k * P + g;
            const double2 x0 = p0[0], x1 = p0[hp], x2 = p0[2 * hp], x3 = p0[3 * hp];
            const double2 w1 = c_conj_if(a.omega[r << sh], conj);
            const double2 w2 = c_conj_if(a.omega[(2 * r) << sh], conj);
            const double2 w3 = c_conj_if(a.omega[(3 * r) << sh], conj);
            const double2 s02 = c_add(x0, x2), d02 = c_sub(x0, x2), s13 = c_add(x1, x3), t = c_sub(x1, x3);
            const double2 d13 = conj ? make_double2(-t.y, t.x) : make_double2(t.y, -t.x);
            p0[0] = c_add(s02, s13);
            p0[hp] = c_mul(c_sub(s02, s13), w2);
            p0[2 * hp] = c_mul(c_add(d02, d13), w1);
            p0[3 * hp] = c_mul(c_sub(d02, d13), w3);
        }
        __syncthreads();
    }

    // ---- store: element (g, t) sits at position brev_L(t)
    const u32 brs = 32 - log_L;
    for (u32 e = threadIdx.x; e < tile; e += kFftThreads) {
        const u32 g = e & (G - 1), t = e >> log_G;
        const u32 pos = log_L ? __brev(t) >> brs : 0;
        double2 v = sm[pos * P + g];
        if constexpr (PASS == 0) {
            // twiddle omega^(k2 t1), k2 = s0 + g < n2, t1 = t < n1 (product < n)
            v = c_mul(v, c_conj_if(a.omega[(s0 + g) * t], conj));
            a.u[(size_t)msg * n + (size_t)t * n2 + s0 + g] = v;
        } else {
            const u32 kk = s0 + g + (t << a.log_n1);   // output index t1 + n1 t2
            if constexpr (MODE == 0) {
                // w_k = u_k zeta^-k / n, rounded to the nearest integers
                const double2 zk = a.zeta[kk];
                const double2 w = c_mul(v, make_double2(zk.x * a.inv_n, -zk.y * a.inv_n));
                const long long lo = __double2ll_rn(w.x), hi = __double2ll_rn(w.y);
                const unsigned long long alo = lo < 0 ? 0ull - (unsigned long long)lo : (unsigned long long)lo;
                const unsigned long long ahi = hi < 0 ? 0ull - (unsigned long long)hi : (unsigned long long)hi;
                u64 *out = a.pt_out + (size_t)msg * a.limbs * 2 * n;
                for (u32 i = 0; i < a.limbs; i++) {
                    const u64 q = a.primes[2 * i], one_sh = a.primes[2 * i + 1];
                    const u64 rl = mul_shoup(alo, 1, one_sh, q), rh = mul_shoup(ahi, 1, one_sh, q);
                    out[(size_t)i * 2 * n + kk] = (lo < 0 && rl) ? q - rl : rl;
                    out[(size_t)i * 2 * n + kk + n] = (hi < 0 && rh) ? q - rh : rh;
                }
            } else {
                a.z_out[(size_t)msg * n + a.slot_of[kk]] = make_double2(v.x * a.scale, v.y * a.scale);
            }
        }
    }
}

// ------------------------------------------------------------- CRT lift

// acc += y * B (NW words each; the caller sizes NW so that nothing carries out).
template <int NW>
__device__ __forceinline__ void mw_mac(u64 (&acc)[NW], u64 y, const u64 *B)
{
    u64 carry = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const u64 b = B[w];
        const u64 lo = y * b, hi = __umul64hi(y, b);
        const u64 s = acc[w] + lo;
        const u64 c1 = s < lo;
        const u64 s2 = s + carry;
        const u64 c2 = s2 < carry;
        acc[w] = s2;
        carry = hi + c1 + c2;
    }
}

// acc -= k * B (two's complement over NW words)
template <int NW>
__device__ __forceinline__ void mw_sub_mul(u64 (&acc)[NW], u64 k, const u64 *B)
{
    u64 borrow = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const u64 b = B[w];
        const u64 lo = k * b, hi = __umul64hi(k, b);
        const u64 d = acc[w] - lo;
        const u64 b1 = acc[w] < lo;
        const u64 d2 = d - borrow;
        const u64 b2 = d < borrow;
        acc[w] = d2;
        borrow = hi + b1 + b2;
    }
}

template <int NW>
__device__ __forceinline__ void mw_add(u64 (&acc)[NW], const u64 *B)
{
    u64 carry = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const u64 s = acc[w] + B[w];
        const u64 c1 = s < B[w];
        const u64 s2 = s + carry;
        carry = c1 + (s2 < carry);
        acc[w] = s2;
    }
}

// Sign of A - B for non-negative NW-word integers (most significant last).
template <int NW>
__device__ __forceinline__ int mw_compare(const u64 (&A)[NW], const u64 *B)
{
    int res = 0;   // decided by the most significant differing word
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const u64 b = B[w];
        if (A[w] != b) res = A[w] > b ? 1 : -1;
    }
    return res;
}

// The nearest double of the signed NW-word integer (round to nearest even):
// the top 64 bits below the leading one, with the lowest bit set when any
// bit further down is set (it lies below the rounding position, so it only
// breaks ties), converted and scaled by a power of two.
template <int NW>
__device__ __forceinline__ double mw_to_double(u64 (&v)[NW])
{
    const bool neg = (long long)v[NW - 1] < 0;
    if (neg) {
        u64 carry = 1;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const u64 x = ~v[w] + carry;
            carry = carry && x == 0;
            v[w] = x;
        }
    }
    int h = -1;
    u64 top = 0, next = 0;
#pragma unroll
    for (int w = 0; w < NW; w++)
        if (v[w]) {
            h = w;
            top = v[w];
            next = w ? v[w - 1] : 0;
        }
    if (h < 0) return 0.0;
    bool sticky = false;
#pragma unroll
    for (int w = 0; w < NW; w++) sticky |= w < h - 1 && v[w] != 0;
    const int lz = __clzll((long long)top);
    u64 m = lz ? (top << lz) | (next >> (64 - lz)) : top;
    sticky |= (lz ? next << lz : next) != 0;
    m |= sticky ? 1u : 0u;
    const double d = ldexp(__ull2double_rn(m), 64 * h - lz);
    return neg ? -d : d;
}

// out[e] = the nearest double of the centred CRT lift of the residues
// coef[(c l + i) N + k] (i < limbs), e = c N + k. Table (level of `limbs`
// primes, NW words per integer): Q, (Q - 1) / 2, Q / q_i for each i, then
// {q_i, [(Q/q_i)^-1]_{q_i}, its Shoup quotient} per i, then the bits of
// 1.0 / (Q / 2^(64 (NW - 2))) as a double. NW = ceil((log2 Q + 6) / 64), so
// that quotient is at least 2^58.
template <int NW>
__global__ void __launch_bounds__(128) k_crt_compose(double *out, const u64 *coef, const u64 *tab, u32 log_N,
                                                     u32 limbs, u64 total)
{
    const u64 *Q = tab, *Qh = tab + NW, *Qhat = tab + 2 * NW, *pr = tab + (2 + limbs) * NW;
    const double inv_qtop = __longlong_as_double((long long)pr[3 * limbs]);
    const u64 N = 1ull << log_N;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 c = e >> log_N, k = e & (N - 1);
        u64 acc[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) acc[w] = 0;
        for (u32 i = 0; i < limbs; i++) {
            const u64 q = pr[3 * i];
            const u64 y = mul_shoup(coef[(c * limbs + i) * N + k], pr[3 * i + 1], pr[3 * i + 2], q);
            mw_mac<NW>(acc, y, Qhat + (size_t)i * NW);
        }
        // acc = x + k Q with 0 <= k < limbs: estimate k from the top two
        // words of acc against Q / 2^(64 (NW - 2)) >= 2^58 (the dropped words
        // and the roundings move it by far less than 1/2), subtract the
        // nearest multiple of Q, and correct the estimate's possible
        // off-by-one exactly
        const double top = fma(__ull2double_rn(acc[NW - 1]), 18446744073709551616.0, __ull2double_rn(acc[NW - 2]));
        mw_sub_mul<NW>(acc, (u64)rint(top * inv_qtop), Q);
        if ((long long)acc[NW - 1] < 0) {
            u64 t[NW];   // t = -acc - 1, and acc < -(Q - 1) / 2 <=> t >= (Q - 1) / 2
#pragma unroll
            for (int w = 0; w < NW; w++) t[w] = ~acc[w];
            if (mw_compare<NW>(t, Qh) >= 0) mw_add<NW>(acc, Q);
        } else if (mw_compare<NW>(acc, Qh) > 0) {
            mw_sub_mul<NW>(acc, 1, Q);
        }
        out[e] = mw_to_double<NW>(acc);
    }
}

// ------------------------------------------------------------- launchers

// 2^10 complex values plus one padding column: below the 48 KB default
static size_t fft_smem(u32 log_L) { return (size_t)((1u << kLogTile) + (1u << log_L)) * sizeof(double2); }

static u32 fft_blocks(const FftArgs &a, u32 log_L)
{
    const u32 log_seqs = a.log_n - log_L;
    const u32 log_G = min(log_seqs, (u32)kLogTile - log_L);
    return a.count << (log_seqs - log_G);
}

template <int MODE>
static cudaError_t fft_two_pass(const FftArgs &a, cudaStream_t s)
{
    const u32 lA = a.log_n1, lB = a.log_n - a.log_n1;
    k_fft_pass<MODE, 0><<<fft_blocks(a, lA), kFftThreads, fft_smem(lA), s>>>(a);
    k_fft_pass<MODE, 1><<<fft_blocks(a, lB), kFftThreads, fft_smem(lB), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_encode_fft(const FftArgs &a, cudaStream_t s) { return fft_two_pass<0>(a, s); }
cudaError_t launch_decode_fft(const FftArgs &a, cudaStream_t s) { return fft_two_pass<1>(a, s); }

#define HE_CRT_NW(X)                                                                                  \
    X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
    X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

u32 crt_words(u32 need) { return need <= 32 ? std::max(need, 2u) : 0; }

cudaError_t launch_crt_compose(double *out, const u64 *coef, const u64 *tab, u32 nw, u32 log_N, u32 limbs, u64 total,
                               u32 blocks, cudaStream_t s)
{
    switch (nw) {
#define HE_CRT_CASE(w)                                                                   \
    case (w):                                                                            \
        k_crt_compose<(w)><<<blocks, 128, 0, s>>>(out, coef, tab, log_N, limbs, total); \
        return cudaGetLastError();
        HE_CRT_NW(HE_CRT_CASE)
#undef HE_CRT_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace he
