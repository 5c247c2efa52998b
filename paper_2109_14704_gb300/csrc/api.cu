// api.cu -- host side of libhe.so: the C ABI declared in include/he.h.
//
// Parameter generation (primes, psi, twiddles, Shoup and Barrett constants)
// runs on the host with 128-bit integer arithmetic; everything on the data
// path runs in the CUDA kernels of kernels.cuh. Argument checks happen before
// anything is enqueued.
#define HE_MISC_KERNELS 1
#include <cuda.h>   // driver types only (CUcontext, CUresult); no link against the driver library
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/he.h"
#include "kernels.cuh"

using he::u32;
using he::u64;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

static he_status fail(he_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

static he_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(HE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HE_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                        \
    } while (0)

extern "C" he_status he_last_error(char *buf, size_t len)
{
    if (!buf || len == 0) return HE_EINVAL;
    size_t n = std::min(len - 1, g_last_error.size());
    memcpy(buf, g_last_error.data(), n);
    buf[n] = 0;
    return HE_OK;
}

extern "C" uint32_t he_version(void) { return 0x000100; }

// --------------------------------------------------------- host arithmetic

static u64 h_mul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

static u64 h_pow(u64 a, u64 e, u64 m)
{
    u64 r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mul(r, a, m);
        a = h_mul(a, a, m);
    }
    return r;
}

static u64 h_inv(u64 a, u64 p) { return h_pow(a % p, p - 2, p); }  // p prime

static u64 shoup(u64 w, u64 p) { return (u64)(((u128)w << 64) / p); }

static int bit_length(u64 x)
{
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// Miller-Rabin with the first twelve primes as witnesses: exact for every
// 64-bit input (Sorenson and Webster, 2015).
static bool h_is_prime(u64 n)
{
    static const u64 W[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 w : W)
        if (n % w == 0) return n == w;
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    for (u64 w : W) {
        u64 x = h_pow(w, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = h_mul(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// The smallest primitive 2N-th root of unity mod q (q prime, 2N | q - 1).
// Odd powers of one primitive root c = g^((q-1)/2N), g a non-residue, run
// over all of them.
static u64 smallest_psi(u64 q, u32 N)
{
    u64 g = 2;
    while (h_pow(g, (q - 1) / 2, q) != q - 1) g++;
    const u64 c = h_pow(g, (q - 1) / (2 * (u64)N), q);
    const u64 c2 = h_mul(c, c, q);
    u64 best = c;
    for (u64 k = 1, x = c; k < N; k++) {
        x = h_mul(x, c2, q);
        if (x < best) best = x;
    }
    return best;
}

static u32 bit_reverse(u32 x, int bits)
{
    u32 r = 0;
    for (int i = 0; i < bits; i++, x >>= 1) r = (r << 1) | (x & 1);
    return r;
}

static int log2_exact(u64 n)
{
    if (n == 0 || (n & (n - 1))) return -1;
    int l = 0;
    while ((1ull << l) < n) l++;
    return l;
}

extern "C" he_status he_primes_generate(uint32_t bits, uint64_t two_n, uint32_t count,
                                        const uint64_t *exclude_host, uint32_t n_exclude,
                                        uint64_t *out_host)
{
    if (bits < 2 || bits > 60) return fail(HE_EINVAL, "bits must be in [2, 60], got %u", bits);
    if (two_n == 0) return fail(HE_EINVAL, "two_n must be positive");
    if (count && !out_host) return fail(HE_EINVAL, "out_host is NULL");
    if (n_exclude && !exclude_host) return fail(HE_EINVAL, "exclude_host is NULL");
    const u64 top = (1ull << bits) - 1, low = 1ull << (bits - 1);
    u64 q = (top - 1) / two_n * two_n + 1;
    u32 got = 0;
    while (got < count && q >= low && q > two_n) {
        bool skip = false;
        for (u32 i = 0; i < n_exclude; i++) skip |= exclude_host[i] == q;
        if (!skip && h_is_prime(q)) out_host[got++] = q;
        q -= two_n;
    }
    if (got < count) return fail(HE_EINVAL, "only %u primes of %u bits = 1 mod %llu", got, bits,
                                 (unsigned long long)two_n);
    return HE_OK;
}

// ------------------------------------------------------------------ tables

// Per-prime constants of the kernels; w1 = psi^-brv(1), the twiddle of the
// last inverse stage.
static he::PrimeConst prime_const(u64 q, u32 N, u64 w1)
{
    he::PrimeConst c;
    memset(&c, 0, sizeof c);
    c.p = q;
    c.two_p = 2 * q;
    c.four_p = 4 * q;
    c.neg_p = 0 - q;
    c.h4 = (u32)((4 * (u128)q + 0xffffffffull) >> 32);
    c.bits = (u32)bit_length(q);
    c.mu = (u64)(((u128)1 << (2 * c.bits + 2)) / q);
    c.ninv = h_inv(N % q, q);
    c.ninv_sh = shoup(c.ninv, q);
    c.w1ninv = h_mul(w1, c.ninv, q);
    c.w1ninv_sh = shoup(c.w1ninv, q);
    c.one_sh = shoup(1, q);
    return c;
}

struct he_ntt_tables {
    u32 N = 0;
    int log_n = 0;
    u32 K = 0;
    std::vector<u64> moduli, psi;
    ulonglong2 *d_fwd = nullptr;  // [K][N] (W, W')
    ulonglong2 *d_inv = nullptr;
    he::PrimeConst *d_pc = nullptr;
};

// the lazy butterfly ranges need 2^30 <= q < 2^60 (Sec. III-A-1: below 60 bits)
static he_status check_modulus_range(u64 q)
{
    if (q < (1ull << 30) || q >= (1ull << 60))
        return fail(HE_EINVAL, "modulus %llu outside [2^30, 2^60)", (unsigned long long)q);
    return HE_OK;
}

static he_status check_modulus(u64 q, u32 N)
{
    if (he_status s = check_modulus_range(q)) return s;
    if ((q - 1) % (2ull * N)) return fail(HE_EINVAL, "modulus %llu is not 1 mod 2N (N = %u)", (unsigned long long)q, N);
    if (!h_is_prime(q)) return fail(HE_EINVAL, "modulus %llu is not prime", (unsigned long long)q);
    return HE_OK;
}

static he_status check_degree(u32 N, int *log_n)
{
    int l = log2_exact(N);
    if (l < 0) return fail(HE_EINVAL, "N = %u is not a power of two", N);
    if (l < 10 || l > 16) return fail(HE_EUNSUPPORTED, "N = %u outside [2^10, 2^16]", N);
    if (!he::degree_ops(l)) return fail(HE_EUNSUPPORTED, "no kernels built for N = %u", N);
    *log_n = l;
    return HE_OK;
}

static void free_tables(he_ntt_tables *t)
{
    if (!t) return;
    cudaFree(t->d_fwd);
    cudaFree(t->d_inv);
    cudaFree(t->d_pc);
    delete t;
}

extern "C" he_status he_ntt_tables_create(uint32_t N, uint32_t limbs, const uint64_t *moduli_host,
                                          he_ntt_tables **out)
{
    if (!out) return fail(HE_EINVAL, "out is NULL");
    *out = nullptr;
    int log_n;
    if (he_status s = check_degree(N, &log_n)) return s;
    if (limbs == 0 || !moduli_host) return fail(HE_EINVAL, "need at least one modulus");
    for (u32 l = 0; l < limbs; l++)
        if (he_status s = check_modulus(moduli_host[l], N)) return s;

    he_ntt_tables *t = new he_ntt_tables;
    t->N = N;
    t->log_n = log_n;
    t->K = limbs;
    t->moduli.assign(moduli_host, moduli_host + limbs);
    std::vector<ulonglong2> fwd((size_t)limbs * N), inv((size_t)limbs * N);
    std::vector<he::PrimeConst> pcs(limbs);
    std::vector<u64> pw(N), pwi(N);
    for (u32 l = 0; l < limbs; l++) {
        const u64 q = moduli_host[l];
        const u64 psi = smallest_psi(q, N), psi_inv = h_inv(psi, q);
        t->psi.push_back(psi);
        pw[0] = pwi[0] = 1;
        for (u32 i = 1; i < N; i++) {
            pw[i] = h_mul(pw[i - 1], psi, q);
            pwi[i] = h_mul(pwi[i - 1], psi_inv, q);
        }
        inv[(size_t)l * N] = make_ulonglong2(1, shoup(1, q));   // k = 0: unused
        for (u32 k = 0; k < N; k++) {
            const u64 w = pw[bit_reverse(k, log_n)], wi = pwi[bit_reverse(k, log_n)];
            fwd[(size_t)l * N + k] = make_ulonglong2(w, shoup(w, q));
            if (k) {
                const int S = 31 - __builtin_clz(k);
                inv[(size_t)l * N + he::inv_tw_pos((int)log_n, S, (int)(k - (1u << S)))] = make_ulonglong2(wi, shoup(wi, q));
            }
        }
        pcs[l] = prime_const(q, N, inv[(size_t)l * N + 1].x);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&t->d_fwd, fwd.size() * sizeof(ulonglong2))) != cudaSuccess ||
        (e = cudaMalloc(&t->d_inv, inv.size() * sizeof(ulonglong2))) != cudaSuccess ||
        (e = cudaMalloc(&t->d_pc, pcs.size() * sizeof(he::PrimeConst))) != cudaSuccess) {
        free_tables(t);
        return fail(HE_ENOMEM, "twiddle tables: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpy(t->d_fwd, fwd.data(), fwd.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(t->d_inv, inv.data(), inv.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(t->d_pc, pcs.data(), pcs.size() * sizeof(he::PrimeConst), cudaMemcpyHostToDevice))) {
        free_tables(t);
        return cuda_fail(e, "upload twiddle tables");
    }
    *out = t;
    return HE_OK;
}

extern "C" he_status he_ntt_tables_destroy(he_ntt_tables *t)
{
    if (t) {
        cudaDeviceSynchronize();
        free_tables(t);
    }
    return HE_OK;
}

extern "C" he_status he_ntt_tables_psi(const he_ntt_tables *t, uint32_t index, uint64_t *psi_out)
{
    if (!t || !psi_out || index >= t->K) return fail(HE_EINVAL, "bad tables, index or output");
    *psi_out = t->psi[index];
    return HE_OK;
}

// ------------------------------------------------------------ transforms

static he_status check_poly_args(const void *poly, uint32_t N, uint32_t limbs, const uint64_t *moduli_host,
                                 const he_ntt_tables *tw, int *log_n)
{
    if (!tw) return fail(HE_EINVAL, "tables are NULL");
    if (he_status s = check_degree(N, log_n)) return s;
    if (tw->N != N) return fail(HE_EINVAL, "tables are for N = %u, not %u", tw->N, N);
    if (limbs > tw->K) return fail(HE_EINVAL, "%u limbs but the tables hold %u primes", limbs, tw->K);
    if (limbs && !moduli_host) return fail(HE_EINVAL, "moduli_host is NULL");
    for (u32 l = 0; l < limbs; l++)
        if (moduli_host[l] != tw->moduli[l])
            return fail(HE_EINVAL, "modulus %u (%llu) differs from the tables' prime (%llu)", l,
                        (unsigned long long)moduli_host[l], (unsigned long long)tw->moduli[l]);
    if (!poly) return fail(HE_EINVAL, "data pointer is NULL");
    if ((uintptr_t)poly & 31) return fail(HE_EINVAL, "data pointer is not 32-byte aligned");
    return HE_OK;
}

static he::NttLaunch uniform_launch(uint64_t *poly, uint32_t limbs, uint32_t count, const he_ntt_tables *tw)
{
    he::NttLaunch a = {};
    a.base = poly;
    a.limbs = limbs;
    a.first_prime = 0;
    a.items = limbs * count;
    a.tw_fwd = tw->d_fwd;
    a.tw_inv = tw->d_inv;
    a.pc = tw->d_pc;
    a.jobs = nullptr;
    return a;
}

// Shape used by he_ntt_fwd / he_ntt_inv per degree (0, 0 = built-in default;
// persistent: a fixed grid walking the limbs instead of one cluster per
// limb), set by he_ntt_set_shape (e.g. from the autotuner).
static std::atomic<int> g_shape_b[2][17], g_shape_e[2][17], g_shape_persistent[2][17];   // [inverse][log N]

// Internally a shape's thread-words code carries the CTAs per SM its
// transform kernels are compiled for in the bits above 4 (inst.cuh).
static int thread_words_code(uint32_t log_thread_words, uint32_t ctas_per_sm)
{
    return (int)(log_thread_words | (ctas_per_sm << 4));
}

extern "C" he_status he_ntt_shapes(uint32_t N, uint32_t *shapes_out, uint32_t cap, uint32_t *n_out)
{
    int log_n;
    if (he_status s = check_degree(N, &log_n)) return s;
    if (!n_out) return fail(HE_EINVAL, "n_out is NULL");
    const he::DegreeOps *ops = he::degree_ops(log_n);
    *n_out = (uint32_t)ops->n_shapes;
    if (cap && !shapes_out) return fail(HE_EINVAL, "shapes_out is NULL");
    for (int i = 0; i < ops->n_shapes && (uint32_t)i < cap; i++) {
        shapes_out[3 * i] = (uint32_t)ops->shapes[i][0];
        shapes_out[3 * i + 1] = (uint32_t)ops->shapes[i][1] & 15u;
        shapes_out[3 * i + 2] = (uint32_t)ops->shapes[i][1] >> 4;
    }
    return HE_OK;
}

extern "C" he_status he_ntt_set_shape(uint32_t N, uint32_t direction, uint32_t log_block,
                                      uint32_t log_thread_words, uint32_t persistent, uint32_t ctas_per_sm)
{
    int log_n;
    if (he_status s = check_degree(N, &log_n)) return s;
    if (direction > 2) return fail(HE_EINVAL, "direction must be 0 (both), 1 (forward) or 2 (inverse)");
    if (log_thread_words > 15 || ctas_per_sm > 32) return fail(HE_EINVAL, "log_thread_words or ctas_per_sm out of range");
    const int code = thread_words_code(log_thread_words, ctas_per_sm);
    if (log_block || code) {
        if (!he::degree_ops(log_n)->has_shape((int)log_block, code))
            return fail(HE_EUNSUPPORTED,
                        "no kernel with 2^%u words per CTA, 2^%u per thread and %u CTAs per SM for N = %u", log_block,
                        log_thread_words, ctas_per_sm, N);
    }
    for (int inv = 0; inv < 2; inv++) {
        if ((direction == 1 && inv) || (direction == 2 && !inv)) continue;
        g_shape_b[inv][log_n].store((int)log_block);
        g_shape_e[inv][log_n].store(code);
        g_shape_persistent[inv][log_n].store(persistent ? 1 : 0);
    }
    return HE_OK;
}

// One launch of a batch of limb transforms in the shape set for the degree.
// cuTensorMapEncodeTiled, fetched through the runtime's driver entry points
// (the library does not link the driver library); null if unavailable.
typedef CUresult (*PfnEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static PfnEncodeTiled encode_tiled()
{
    static std::once_flag once;
    static PfnEncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PfnEncodeTiled)f;
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a uniform batch for the forward transform's bulk stores:
// the items N words at base as rows of 16 words (128 bytes, the row stride),
// boxes of 32 rows (one warp's output), 128-byte swizzle. false (plain
// stores) if the encoder is unavailable, base is not 128-byte aligned, or
// the batch has 2^32 rows or more.
static bool batch_tmap(he::NttLaunch &a, u32 N)
{
    PfnEncodeTiled enc = encode_tiled();
    if (!enc || a.jobs || ((uintptr_t)a.base & 127)) return false;
    const cuuint64_t rows = (cuuint64_t)a.items * N / 16;
    if (rows < 32 || rows >= (1ull << 32)) return false;
    const cuuint64_t dims[2] = {16, rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {16, 32};
    const cuuint32_t estr[2] = {1, 1};
    return enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, a.base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static he_status ntt_launch(const he::NttLaunch &a0, int log_n, bool inv, cudaStream_t stream)
{
    const he::DegreeOps *ops = he::degree_ops(log_n);
    const int lb = g_shape_b[inv][log_n].load(), le = g_shape_e[inv][log_n].load();
    he::NttLaunch a = a0;
    const u32 resident = (u32)std::max(ops->max_clusters(lb, le, inv), 1);
#ifndef HE_NO_L2_PREFETCH
    a.prefetch = a.items > resident ? resident : 0;   // persistent form: any non-zero value
#else
    a.prefetch = 0;
#endif
    if (g_shape_persistent[inv][log_n].load()) {
        HE_CUDA(ops->ntt_persistent(a, lb, le, inv, std::min<u32>(a.items, resident), stream));
    } else {
        a.tma_store = (!inv && le == 4 && batch_tmap(a, 1u << log_n)) ? 1u : 0u;
        HE_CUDA(ops->ntt(a, lb, le, inv, stream));
    }
    return HE_OK;
}

static he_status ntt_common(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                            const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream, bool inv)
{
    int log_n;
    if (he_status s = check_poly_args(poly, N, limbs, moduli_host, tw, &log_n)) return s;
    if ((u64)limbs * count == 0) return HE_OK;
    if ((u64)limbs * count * (N / 4096 + 1) > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
    return ntt_launch(uniform_launch(poly, limbs, count, tw), log_n, inv, (cudaStream_t)stream);
}

extern "C" he_status he_ntt_fwd(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                                const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream)
{
    return ntt_common(poly, N, limbs, count, moduli_host, tw, stream, false);
}

extern "C" he_status he_ntt_inv(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                                const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream)
{
    return ntt_common(poly, N, limbs, count, moduli_host, tw, stream, true);
}

static he_status naive_common(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                              const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream, bool inv)
{
    int log_n;
    if (he_status s = check_poly_args(poly, N, limbs, moduli_host, tw, &log_n)) return s;
    if ((u64)limbs * count == 0) return HE_OK;
    const he::NttLaunch a = uniform_launch(poly, limbs, count, tw);
    const u64 bfly = (u64)a.items * (N / 2);
    const u32 threads = 256;
    const u32 grid = (u32)((bfly + threads - 1) / threads);
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < log_n; k++) {
        const u32 S = inv ? (u32)(log_n - 1 - k) : (u32)k;
        he::k_ntt_naive_stage<<<grid, threads, 0, s>>>(a, (u32)log_n, S, inv);
    }
    if (!inv) {
        const u32 g2 = (u32)(((u64)a.items * N + threads - 1) / threads);
        he::k_ntt_naive_final<<<g2, threads, 0, s>>>(a, (u32)log_n);
    }
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

extern "C" he_status he_ntt_fwd_naive(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                                      const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream)
{
    return naive_common(poly, N, limbs, count, moduli_host, tw, stream, false);
}

extern "C" he_status he_ntt_inv_naive(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                                      const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream)
{
    return naive_common(poly, N, limbs, count, moduli_host, tw, stream, true);
}

static int g_num_sms = 0;

static int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_num_sms = 152;
    }
    return g_num_sms;
}

static u32 stream_grid(u64 work_items, u32 threads)
{
    const u64 want = (work_items + threads - 1) / threads;
    const u64 cap = (u64)num_sms() * 8;
    return (u32)std::max<u64>(1, std::min(want, cap));
}

extern "C" he_status he_dyadic_mul(uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t N,
                                   uint32_t limbs, uint32_t count, const uint64_t *moduli_host,
                                   const he_ntt_tables *tw, he_stream_t stream)
{
    int log_n;
    if (he_status s = check_poly_args(out, N, limbs, moduli_host, tw, &log_n)) return s;
    if (!a || !b || ((uintptr_t)a & 31) || ((uintptr_t)b & 31))
        return fail(HE_EINVAL, "inputs must be non-NULL and 32-byte aligned");
    const u64 items = (u64)limbs * count;
    if (!items) return HE_OK;
    he::k_dyadic<<<stream_grid(items * N / 2, 256), 256, 0, (cudaStream_t)stream>>>(
        out, a, b, (u32)log_n, (u32)items, limbs, 0, tw->d_pc);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

extern "C" he_status he_negacyclic_mul(uint64_t *c, const uint64_t *a, const uint64_t *b, uint32_t N,
                                       uint32_t limbs, uint32_t count, const uint64_t *moduli_host,
                                       const he_ntt_tables *tw, he_stream_t stream)
{
    int log_n;
    if (he_status s = check_poly_args(c, N, limbs, moduli_host, tw, &log_n)) return s;
    if (!a || !b || ((uintptr_t)a & 31) || ((uintptr_t)b & 31))
        return fail(HE_EINVAL, "inputs must be non-NULL and 32-byte aligned");
    const u64 items = (u64)limbs * count;
    if (!items) return HE_OK;
    if (items * (N / 4096 + 1) > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
    const u64 words = items * N;
    const uintptr_t cb = (uintptr_t)c, ce = cb + words * 8;
    for (const uint64_t *in : {a, b})
        if ((uintptr_t)in < ce && cb < (uintptr_t)in + words * 8 && (uintptr_t)in != cb)
            return fail(HE_EINVAL, "c overlaps an input without being equal to it");
    // c may equal a or b: each cluster reads its limb of both before it writes c
    he::NegaLaunch L = {};
    L.c = c;
    L.a = a;
    L.b = b;
    L.limbs = limbs;
    L.items = (u32)items;
    L.tw_fwd = tw->d_fwd;
    L.tw_inv = tw->d_inv;
    L.pc = tw->d_pc;
    HE_CUDA(he::degree_ops(log_n)->negacyclic(L, g_shape_b[0][log_n].load(), g_shape_e[0][log_n].load(),
                                              (cudaStream_t)stream));
    return HE_OK;
}

// ----------------------------------------------------------------- context

struct he_context {
    u32 N = 0;
    int log_n = 0;
    u32 n_data = 0;
    std::vector<u64> data;
    u64 P = 0;
    he_ntt_tables *tables = nullptr;   // primes q_0..q_L, P
    u64 *d_cst = nullptr;
    std::atomic<int> eval_log_e{4};    // words per thread of the evaluation kernels
};

struct he_relin_key {
    const he_context *ctx = nullptr;
    ulonglong2 *d_evk = nullptr;
};

extern "C" he_status he_context_create(uint32_t N, uint32_t n_data, const uint64_t *data_moduli_host,
                                       uint64_t special_modulus, he_context **out)
{
    if (!out) return fail(HE_EINVAL, "out is NULL");
    *out = nullptr;
    int log_n;
    if (he_status s = check_degree(N, &log_n)) return s;
    if (n_data < 1 || n_data > 32) return fail(HE_EINVAL, "n_data must be in [1, 32], got %u", n_data);
    if (!data_moduli_host) return fail(HE_EINVAL, "data_moduli_host is NULL");
    std::vector<u64> all(data_moduli_host, data_moduli_host + n_data);
    all.push_back(special_modulus);
    for (size_t i = 0; i < all.size(); i++) {
        if (he_status s = check_modulus(all[i], N)) return s;
        // key switching reduces words below 2^60 modulo every prime with one
        // Barrett step, which needs q >= 2^31
        if (all[i] < (1ull << 30)) return fail(HE_EINVAL, "modulus %llu has fewer than 31 bits", (unsigned long long)all[i]);
        for (size_t j = 0; j < i; j++)
            if (all[j] == all[i]) return fail(HE_EINVAL, "modulus %llu appears twice", (unsigned long long)all[i]);
    }
    he_context *c = new he_context;
    c->N = N;
    c->log_n = log_n;
    c->n_data = n_data;
    c->data.assign(data_moduli_host, data_moduli_host + n_data);
    c->P = special_modulus;
    if (he_status s = he_ntt_tables_create(N, n_data + 1, all.data(), &c->tables)) {
        delete c;
        return s;
    }
    std::vector<u64> cst(3 * (size_t)n_data + 3 * (size_t)n_data * n_data + n_data, 0);
    for (u32 i = 0; i < n_data; i++) {
        const u64 q = all[i];
        cst[3 * i + 0] = h_inv(special_modulus % q, q);
        cst[3 * i + 1] = shoup(cst[3 * i + 0], q);
        cst[3 * i + 2] = special_modulus % q;
        cst[3 * (size_t)n_data * (1 + n_data) + i] = shoup(special_modulus % q, q);
    }
    for (u32 l = 1; l < n_data; l++)
        for (u32 i = 0; i < l; i++) {
            const u64 q = all[i], ql = all[l];
            u64 *d = &cst[3 * n_data + 3 * ((size_t)l * n_data + i)];
            d[0] = h_inv(ql % q, q);
            d[1] = shoup(d[0], q);
            d[2] = ql % q;
        }
    cudaError_t e = cudaMalloc(&c->d_cst, cst.size() * sizeof(u64));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_cst, cst.data(), cst.size() * sizeof(u64), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        he_ntt_tables_destroy(c->tables);
        cudaFree(c->d_cst);
        delete c;
        return cuda_fail(e, "context constants");
    }
    *out = c;
    return HE_OK;
}

extern "C" he_status he_context_set_eval_shape(he_context *ctx, uint32_t log_thread_words)
{
    if (!ctx) return fail(HE_EINVAL, "context is NULL");
    if (log_thread_words != 0 && log_thread_words != 3 && log_thread_words != 4)
        return fail(HE_EUNSUPPORTED, "evaluation kernels are built with 2^3 or 2^4 words per thread");
    ctx->eval_log_e.store(log_thread_words ? (int)log_thread_words : 4);
    return HE_OK;
}

extern "C" he_status he_context_destroy(he_context *ctx)
{
    if (ctx) {
        cudaDeviceSynchronize();
        he_ntt_tables_destroy(ctx->tables);
        cudaFree(ctx->d_cst);
        delete ctx;
    }
    return HE_OK;
}

extern "C" he_status he_relin_key_upload(const he_context *ctx, const uint64_t *evk_host, he_relin_key **out)
{
    if (!out) return fail(HE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx || !evk_host) return fail(HE_EINVAL, "context or key is NULL");
    const u32 nd = ctx->n_data, N = ctx->N;
    const size_t words = (size_t)nd * 2 * (nd + 1) * N;
    std::vector<ulonglong2> dev(words);
    for (u32 j = 0; j < nd; j++)
        for (u32 k = 0; k < 2; k++)
            for (u32 t = 0; t <= nd; t++) {
                const u64 q = ctx->tables->moduli[t];
                const size_t base = (((size_t)j * 2 + k) * (nd + 1) + t) * N;
                for (u32 i = 0; i < N; i++) {
                    const u64 w = evk_host[base + i];
                    if (w >= q) return fail(HE_EINVAL, "key word %zu is not reduced mod its prime", base + i);
                    dev[base + i] = make_ulonglong2(w, shoup(w, q));
                }
            }
    he_relin_key *key = new he_relin_key;
    key->ctx = ctx;
    cudaError_t e = cudaMalloc(&key->d_evk, words * sizeof(ulonglong2));
    if (e == cudaSuccess) e = cudaMemcpy(key->d_evk, dev.data(), words * sizeof(ulonglong2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(key->d_evk);
        delete key;
        return fail(e == cudaErrorMemoryAllocation ? HE_ENOMEM : HE_ECUDA, "relin key upload: %s",
                    cudaGetErrorString(e));
    }
    *out = key;
    return HE_OK;
}

extern "C" he_status he_relin_key_destroy(he_relin_key *key)
{
    if (key) {
        cudaDeviceSynchronize();
        cudaFree(key->d_evk);
        delete key;
    }
    return HE_OK;
}

static he::DevCtx dev_ctx(const he_context *c)
{
    he::DevCtx d;
    d.tw_fwd = c->tables->d_fwd;
    d.tw_inv = c->tables->d_inv;
    d.pc = c->tables->d_pc;
    d.cst = c->d_cst;
    d.N = c->N;
    d.n_data = c->n_data;
    return d;
}

static he_status check_ptr(const void *p, const char *name)
{
    if (!p) return fail(HE_EINVAL, "%s is NULL", name);
    if ((uintptr_t)p & 31) return fail(HE_EINVAL, "%s is not 32-byte aligned", name);
    return HE_OK;
}

static he_status check_level(const he_context *ctx, uint32_t level, bool need_rescale)
{
    if (!ctx) return fail(HE_EINVAL, "context is NULL");
    if (level >= ctx->n_data) return fail(HE_EINVAL, "level %u >= number of data primes %u", level, ctx->n_data);
    if (need_rescale && level < 1) return fail(HE_EINVAL, "rescale needs level >= 1");
    return HE_OK;
}

extern "C" he_status he_ct_mul(uint64_t *out3, const uint64_t *ct_a, const uint64_t *ct_b, const he_context *ctx,
                               uint32_t level, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (he_status s = check_ptr(out3, "out3")) return s;
    if (he_status s = check_ptr(ct_a, "ct_a")) return s;
    if (he_status s = check_ptr(ct_b, "ct_b")) return s;
    const u32 n = level + 1;
    he::k_tensor<<<stream_grid((u64)n * ctx->N / 2, 256), 256, 0, (cudaStream_t)stream>>>(
        out3, ct_a, ct_b, (u32)ctx->log_n, n, 1, ctx->tables->d_pc);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// Scratch of key switching and rescale, in words per ciphertext (the
// minimum, with the fused mod-up), plus the expanded mod-up's buffer for a
// group of ciphertexts.
static size_t relin_words(const he_context *c, u32 n) { return (size_t)(3 * n + 2) * c->N; }
static size_t rescale_words(const he_context *c) { return (size_t)2 * c->N; }
static size_t mrr_words(const he_context *c, u32 n) { return (size_t)(3 * n + 4) * c->N; }
static const u32 kModupGroup = 64;  // ciphertexts per expanded mod-up group (fewer, larger launches)
static size_t modup_x_words(const he_context *c, u32 n, u32 group) { return (size_t)group * (n + 1) * n * c->N; }

extern "C" size_t he_relin_scratch_bytes(const he_context *ctx, uint32_t level)
{
    return ctx ? (relin_words(ctx, level + 1) + modup_x_words(ctx, level + 1, 1)) * 8 : 0;
}

extern "C" size_t he_rescale_scratch_bytes(const he_context *ctx, uint32_t level)
{
    (void)level;
    return ctx ? rescale_words(ctx) * 8 : 0;
}

extern "C" size_t he_mul_relin_rescale_scratch_bytes_ex(const he_context *ctx, uint32_t level, uint32_t count,
                                                        uint32_t expand_group)
{
    if (!ctx || !count) return 0;
    const u32 group = std::min({count, kModupGroup, expand_group});
    return (mrr_words(ctx, level + 1) * count + modup_x_words(ctx, level + 1, group)) * 8;
}

extern "C" size_t he_mul_relin_rescale_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count)
{
    return he_mul_relin_rescale_scratch_bytes_ex(ctx, level, count, kModupGroup);
}

static he_status run_eval(const he_context *ctx, he::EvalKernel k, const he::EvalArgs &a, u32 items,
                          cudaStream_t s, const he::JobTable *jobs = nullptr)
{
    if (!items) return HE_OK;
    HE_CUDA(he::degree_ops(ctx->log_n)->eval(k, a, items, ctx->eval_log_e.load(), jobs, s));
    return HE_OK;
}

// The special prime's accumulators of `limbs` back-to-back N-word rows at
// `plift` go through the inverse transform in place.
static he_status plift_intt(const he_context *ctx, u64 *plift, u32 limbs, cudaStream_t s)
{
    he::NttLaunch L = {};
    L.base = plift;
    L.limbs = 1;
    L.first_prime = ctx->n_data;
    L.items = limbs;
    L.tw_fwd = ctx->tables->d_fwd;
    L.tw_inv = ctx->tables->d_inv;
    L.pc = ctx->tables->d_pc;
    return ntt_launch(L, ctx->log_n, true, s);
}

// Mod-up of key switching for `count` ciphertexts (a.c2 holds their
// coefficient-domain digits): accq and plift as k_ks_modup leaves them.
// With room for the expanded buffer (x_words at xbuf, at least one
// ciphertext's (n + 1) n N words) the transforms run as independent plain-
// size launches (k_ks_expand), the key products as an elementwise pass
// (k_ks_mac) and the special prime's accumulators go through the inverse
// transform in place; the buffer takes groups of up to kModupGroup
// ciphertexts. Otherwise the fused k_ks_modup runs.
// The tiled key multiply-accumulate's shared memory, 2 n MAC_TILE key pairs
// (64 KB at the largest chain, n = 32), above the default 48 KB limit.
static cudaError_t mac_tiled_smem_attr()
{
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        e = cudaFuncSetAttribute(he::k_ks_mac_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * 32 * he::MAC_TILE * sizeof(ulonglong2)));
    });
    return e;
}

static he_status ks_modup(const he_context *ctx, he::EvalArgs &a, u32 count, u64 *xbuf, size_t x_words,
                          cudaStream_t s)
{
    const u32 n = a.n;
    const size_t per = (size_t)(n + 1) * n * ctx->N;
    const u32 group = (u32)std::min<size_t>({(size_t)kModupGroup, (size_t)count, xbuf ? x_words / per : 0});
    if (group == 0) return run_eval(ctx, he::EK_KS_MODUP, a, count * (n + 1), s);
    a.mx = xbuf;
    for (u32 c0 = 0; c0 < count; c0 += group) {
        const u32 gs = std::min(group, count - c0);
        a.c_first = c0;
        if (he_status r = run_eval(ctx, he::EK_KS_EXPAND, a, gs * (n + 1) * n, s)) return r;
        if (gs >= 8) {   // every ciphertext lane of the tiled kernel busy
            const u32 blocks = (n + 1) * (ctx->N / he::MAC_TILE) * ((gs + he::MAC_CHUNK - 1) / he::MAC_CHUNK);
            const u32 smem = n * 2 * he::MAC_TILE * (u32)sizeof(ulonglong2);
            if (cudaError_t e = mac_tiled_smem_attr()) return cuda_fail(e, "k_ks_mac_tiled attribute");
            he::k_ks_mac_tiled<<<blocks, 256, smem, s>>>(a, gs);
        } else {
            const u32 total = (u32)((gs + he::MAC_CTS - 1) / he::MAC_CTS * (n + 1) * (ctx->N / 2));
            he::k_ks_mac<false><<<stream_grid(total, 256), 256, 0, s>>>(a, gs, total, he::NoJobs{});
        }
        HE_CUDA(cudaGetLastError());
    }
    a.mx = nullptr;
    a.c_first = 0;
    return plift_intt(ctx, a.plift, 2 * count, s);
}

extern "C" he_status he_relin(uint64_t *ct_out2, const uint64_t *ct_in3, const he_relin_key *key,
                              const he_context *ctx, uint32_t level, void *scratch, size_t scratch_bytes,
                              he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (!key || key->ctx != ctx) return fail(HE_EINVAL, "relin key is NULL or belongs to another context");
    if (he_status s = check_ptr(ct_out2, "ct_out2")) return s;
    if (he_status s = check_ptr(ct_in3, "ct_in3")) return s;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    const u32 n = level + 1;
    if (scratch_bytes < relin_words(ctx, n) * 8) return fail(HE_EINVAL, "scratch too small");
    he::EvalArgs a = {};
    a.ct3 = ct_in3;
    a.out = ct_out2;
    a.c2 = (u64 *)scratch;
    a.accq = a.c2 + (size_t)n * ctx->N;
    a.plift = a.accq + (size_t)2 * n * ctx->N;
    a.evk = key->d_evk;
    a.n = n;
    a.count = 1;
    a.ctx = dev_ctx(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    u64 *xbuf = (u64 *)scratch + relin_words(ctx, n);
    const size_t x_words = scratch_bytes / 8 - relin_words(ctx, n);
    if (he_status r = run_eval(ctx, he::EK_KS_DIGITS, a, n, s)) return r;
    if (he_status r = ks_modup(ctx, a, 1, xbuf, x_words, s)) return r;
    return run_eval(ctx, he::EK_KS_MODDOWN, a, 2 * n, s);
}

extern "C" he_status he_rescale(uint64_t *ct_out, const uint64_t *ct_in, const he_context *ctx, uint32_t level,
                                void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, true)) return s;
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (he_status s = check_ptr(ct_in, "ct_in")) return s;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < rescale_words(ctx) * 8) return fail(HE_EINVAL, "scratch too small");
    he::EvalArgs a = {};
    a.ct2 = ct_in;
    a.out = ct_out;
    a.lift2 = (u64 *)scratch;
    a.n = level + 1;
    a.count = 1;
    a.ctx = dev_ctx(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (he_status r = run_eval(ctx, he::EK_RS_LIFT, a, 2, s)) return r;
    return run_eval(ctx, he::EK_RS, a, 2 * level, s);
}

// Key switching of `count` ciphertexts whose third component is given either
// as the tensor of a pair (ct_a, ct_b: Mul fused into the loads) or as a
// three-component input ct3, then (rescale = true) RS by q_l (MulLinRS
// kernels) or (rescale = false) the mod-down only (MulLin / Relin).
static he_status key_switch_common(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b, const uint64_t *ct3,
                                   uint32_t count, const he_relin_key *key, const he_context *ctx, uint32_t level,
                                   void *scratch, size_t scratch_bytes, he_stream_t stream, bool rescale)
{
    if (he_status s = check_level(ctx, level, rescale)) return s;
    if (!key || key->ctx != ctx) return fail(HE_EINVAL, "relin key is NULL or belongs to another context");
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (ct3) {
        if (he_status s = check_ptr(ct3, "ct3")) return s;
    } else {
        if (he_status s = check_ptr(ct_a, "ct_a")) return s;
        if (he_status s = check_ptr(ct_b, "ct_b")) return s;
    }
    if (count == 0) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    const u32 n = level + 1;
    const size_t base_words = (rescale ? mrr_words(ctx, n) : relin_words(ctx, n)) * count;
    if (scratch_bytes < base_words * 8) return fail(HE_EINVAL, "scratch too small");
    if ((u64)count * 2 * n * (ctx->N / 4096 + 1) > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
    he::EvalArgs a = {};
    a.ct_a = ct3 ? nullptr : ct_a;
    a.ct_b = ct3 ? nullptr : ct_b;
    a.ct3 = ct3;
    a.out = ct_out;
    a.c2 = (u64 *)scratch;
    a.accq = a.c2 + (size_t)count * n * ctx->N;
    a.plift = a.accq + (size_t)count * 2 * n * ctx->N;
    a.lift2 = rescale ? a.plift + (size_t)count * 2 * ctx->N : nullptr;
    a.evk = key->d_evk;
    a.n = n;
    a.count = count;
    a.ctx = dev_ctx(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    u64 *xbuf = (u64 *)scratch + base_words;
    const size_t x_words = scratch_bytes / 8 - base_words;
    if (he_status r = run_eval(ctx, he::EK_KS_DIGITS, a, count * n, s)) return r;
    if (he_status r = ks_modup(ctx, a, count, xbuf, x_words, s)) return r;
    if (!rescale) return run_eval(ctx, he::EK_KS_MODDOWN, a, count * 2 * n, s);
    if (he_status r = run_eval(ctx, he::EK_MRR_LAST, a, count * 2, s)) return r;
    if (he_status r = run_eval(ctx, he::EK_MRR_REST_Z, a, count * 2 * level, s)) return r;
    return run_eval(ctx, he::EK_MRR_REST_OUT, a, count * 2 * level, s);
}

extern "C" he_status he_mul_relin_rescale(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b,
                                          uint32_t count, const he_relin_key *key, const he_context *ctx,
                                          uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    return key_switch_common(ct_out, ct_a, ct_b, nullptr, count, key, ctx, level, scratch, scratch_bytes, stream,
                             true);
}

extern "C" he_status he_sqr_relin_rescale(uint64_t *ct_out, const uint64_t *ct_a, uint32_t count,
                                          const he_relin_key *key, const he_context *ctx, uint32_t level,
                                          void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    return key_switch_common(ct_out, ct_a, ct_a, nullptr, count, key, ctx, level, scratch, scratch_bytes, stream,
                             true);
}

extern "C" he_status he_relin_rescale(uint64_t *ct_out, const uint64_t *ct3, uint32_t count,
                                      const he_relin_key *key, const he_context *ctx, uint32_t level, void *scratch,
                                      size_t scratch_bytes, he_stream_t stream)
{
    if (!ct3) return fail(HE_EINVAL, "ct3 is NULL");
    return key_switch_common(ct_out, nullptr, nullptr, ct3, count, key, ctx, level, scratch, scratch_bytes, stream,
                             true);
}

// ---- mixed-level MulLinRS batches (one launch per pipeline stage) -----------

// Scratch words of one job of a mixed batch: c2, accq, lift2, the expanded
// mod-up buffer of all its ciphertexts, and its share of the common plift.
static size_t mrr_job_words(const he_context *c, u32 n, u32 count)
{
    return ((size_t)n + 2 * n + 2 + (size_t)(n + 1) * n + 2) * c->N * count;
}

// Levels and counts of every job; with `pointers`, also each live job's buffers.
static he_status check_mrr_jobs(const he_context *ctx, const he_mrr_job *jobs, uint32_t n_jobs, bool pointers)
{
    if (!ctx) return fail(HE_EINVAL, "context is NULL");
    if (n_jobs && !jobs) return fail(HE_EINVAL, "jobs_host is NULL");
    for (u32 i = 0; i < n_jobs; i++) {
        const he_mrr_job &J = jobs[i];
        if (he_status s = check_level(ctx, J.level, true)) return s;
        if (J.count > 4096) return fail(HE_EINVAL, "job %u: more than 4096 ciphertext pairs", i);
        if (!J.count || !pointers) continue;
        if (he_status s = check_ptr(J.ct_out, "ct_out")) return s;
        if (he_status s = check_ptr(J.ct_a, "ct_a")) return s;
        if (he_status s = check_ptr(J.ct_b, "ct_b")) return s;
    }
    return HE_OK;
}

extern "C" size_t he_mul_relin_rescale_batch_scratch_bytes(const he_context *ctx, const he_mrr_job *jobs_host,
                                                           uint32_t n_jobs)
{
    if (check_mrr_jobs(ctx, jobs_host, n_jobs, false) != HE_OK) return 0;
    size_t words = 0;
    for (u32 i = 0; i < n_jobs; i++) words += mrr_job_words(ctx, jobs_host[i].level + 1, jobs_host[i].count);
    return words * 8;
}

// One pass of the pipeline over up to kMaxJobs jobs whose scratch starts at w.
static he_status mrr_jobs_pass(const he_mrr_job *jobs, u32 n_jobs, const he_relin_key *key, const he_context *ctx,
                               u64 *w, cudaStream_t s)
{
    he::JobTable t = {};
    u64 tot[he::JS_COUNT] = {};
    u32 pairs = 0;
    for (u32 i = 0; i < n_jobs; i++) pairs += jobs[i].count;
    u64 *plift = w;                       // [all pairs][2][N], contiguous for one transform launch
    w += (size_t)pairs * 2 * ctx->N;
    u64 *pl = plift;
    for (u32 i = 0; i < n_jobs; i++) {
        const he_mrr_job &J = jobs[i];
        const u32 n = J.level + 1, c = J.count;
        he::EvalJob &E = t.job[t.n_jobs++];
        E.ct_a = J.ct_a;
        E.ct_b = J.ct_b;
        E.out = J.ct_out;
        E.n = n;
        E.count = c;
        E.c2 = w;
        E.accq = E.c2 + (size_t)c * n * ctx->N;
        E.lift2 = E.accq + (size_t)c * 2 * n * ctx->N;
        E.mx = E.lift2 + (size_t)c * 2 * ctx->N;
        w = E.mx + (size_t)c * (n + 1) * n * ctx->N;
        E.plift = pl;
        pl += (size_t)c * 2 * ctx->N;
        E.evk = key->d_evk;
        E.ctx = dev_ctx(ctx);
        const u64 items[he::JS_COUNT] = {(u64)c * n, (u64)c * (n + 1) * n,
                                         (u64)(c + he::MAC_CTS - 1) / he::MAC_CTS * (n + 1) * (ctx->N / 2), 2ull * c,
                                         2ull * c * (n - 1)};
        for (int st = 0; st < he::JS_COUNT; st++) {
            if (tot[st] + items[st] > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
            E.begin[st] = (u32)tot[st];
            tot[st] += items[st];
        }
    }
    u64 grid_items = 0;
    for (int st = 0; st < he::JS_COUNT; st++) grid_items = std::max<u64>(grid_items, tot[st]);
    if (grid_items * 8 > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
    he::EvalArgs a = {};
    a.evk = key->d_evk;
    a.ctx = dev_ctx(ctx);
    a.n = t.job[0].n;   // unused with a job table; kept valid
    if (he_status r = run_eval(ctx, he::EK_KS_DIGITS, a, (u32)tot[he::JS_DIGITS], s, &t)) return r;
    if (he_status r = run_eval(ctx, he::EK_KS_EXPAND, a, (u32)tot[he::JS_EXPAND], s, &t)) return r;
    he::k_ks_mac<true><<<stream_grid(tot[he::JS_MAC], 256), 256, 0, s>>>(a, 0, (u32)tot[he::JS_MAC], t);
    HE_CUDA(cudaGetLastError());
    if (he_status r = plift_intt(ctx, plift, 2 * pairs, s)) return r;
    if (he_status r = run_eval(ctx, he::EK_MRR_LAST, a, (u32)tot[he::JS_LAST], s, &t)) return r;
    if (he_status r = run_eval(ctx, he::EK_MRR_REST_Z, a, (u32)tot[he::JS_REST], s, &t)) return r;
    return run_eval(ctx, he::EK_MRR_REST_OUT, a, (u32)tot[he::JS_REST], s, &t);
}

extern "C" he_status he_mul_relin_rescale_batch(const he_mrr_job *jobs_host, uint32_t n_jobs,
                                                const he_relin_key *key, const he_context *ctx, void *scratch,
                                                size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_mrr_jobs(ctx, jobs_host, n_jobs, true)) return s;
    if (!key || key->ctx != ctx) return fail(HE_EINVAL, "relin key is NULL or belongs to another context");
    std::vector<he_mrr_job> live;
    for (u32 i = 0; i < n_jobs; i++)
        if (jobs_host[i].count) live.push_back(jobs_host[i]);
    if (live.empty()) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < he_mul_relin_rescale_batch_scratch_bytes(ctx, live.data(), (u32)live.size()))
        return fail(HE_EINVAL, "scratch too small");
    u64 *w = (u64 *)scratch;
    for (size_t i = 0; i < live.size(); i += he::kMaxJobs) {
        const u32 m = (u32)std::min<size_t>(he::kMaxJobs, live.size() - i);
        if (he_status r = mrr_jobs_pass(live.data() + i, m, key, ctx, w, (cudaStream_t)stream)) return r;
        for (u32 k = 0; k < m; k++) w += mrr_job_words(ctx, live[i + k].level + 1, live[i + k].count);
    }
    return HE_OK;
}

extern "C" size_t he_mul_relin_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count)
{
    if (!ctx || !count) return 0;
    return (relin_words(ctx, level + 1) * count + modup_x_words(ctx, level + 1, std::min(count, kModupGroup))) * 8;
}

extern "C" he_status he_mul_relin(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b, uint32_t count,
                                  const he_relin_key *key, const he_context *ctx, uint32_t level, void *scratch,
                                  size_t scratch_bytes, he_stream_t stream)
{
    return key_switch_common(ct_out, ct_a, ct_b, nullptr, count, key, ctx, level, scratch, scratch_bytes, stream,
                             false);
}

extern "C" he_status he_ct_add(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b, uint32_t count,
                               uint32_t components, const he_context *ctx, uint32_t level, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (components != 2 && components != 3) return fail(HE_EINVAL, "components must be 2 or 3, got %u", components);
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (he_status s = check_ptr(ct_a, "ct_a")) return s;
    if (he_status s = check_ptr(ct_b, "ct_b")) return s;
    if (count == 0) return HE_OK;
    const u32 n = level + 1;
    const u64 words = (u64)count * components * n * ctx->N;
    he::k_ct_add<<<stream_grid(words / 2, 256), 256, 0, (cudaStream_t)stream>>>(
        ct_out, ct_a, ct_b, words, (u32)ctx->log_n, n, ctx->tables->d_pc);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

static he_status check_galois(const he_context *ctx, uint32_t g)
{
    if (!(g & 1) || g >= 2 * ctx->N) return fail(HE_EINVAL, "Galois element %u is not odd and below 2N = %u", g, 2 * ctx->N);
    return HE_OK;
}

extern "C" he_status he_ct_automorph(uint64_t *ct_out, const uint64_t *ct_in, uint32_t count, uint32_t components,
                                     uint32_t galois_elt, const he_context *ctx, uint32_t level, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (he_status s = check_galois(ctx, galois_elt)) return s;
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (he_status s = check_ptr(ct_in, "ct_in")) return s;
    if (ct_out == ct_in) return fail(HE_EINVAL, "the automorphism cannot work in place");
    if (count == 0 || components == 0) return HE_OK;
    const u64 words = (u64)count * components * (level + 1) * ctx->N;
    he::k_ct_automorph<<<stream_grid(words, 256), 256, 0, (cudaStream_t)stream>>>(ct_out, ct_in, words,
                                                                                  (u32)ctx->log_n, galois_elt);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// Rotate scratch: the three-component input (sigma(c0), 0, sigma(c1)) of the
// key switch, then the key switch's own scratch (with the expanded mod-up).
static size_t rotate_c3_words(const he_context *c, u32 n, u32 count) { return (size_t)3 * n * c->N * count; }

extern "C" size_t he_rotate_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count)
{
    if (!ctx || !count) return 0;
    return rotate_c3_words(ctx, level + 1, count) * 8 + he_mul_relin_scratch_bytes(ctx, level, count);
}

extern "C" he_status he_rotate(uint64_t *ct_out, const uint64_t *ct_in, uint32_t count, uint32_t galois_elt,
                               const he_relin_key *galois_key, const he_context *ctx, uint32_t level, void *scratch,
                               size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (he_status s = check_galois(ctx, galois_elt)) return s;
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (he_status s = check_ptr(ct_in, "ct_in")) return s;
    if (count == 0) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    const u32 n = level + 1;
    const size_t c3_words = rotate_c3_words(ctx, n, count);
    if (scratch_bytes < (c3_words + relin_words(ctx, n) * count) * 8) return fail(HE_EINVAL, "scratch too small");
    u64 *c3 = (u64 *)scratch;
    const size_t comp = (size_t)n * ctx->N;
    cudaStream_t s = (cudaStream_t)stream;
    // (sigma(c0), 0, sigma(c1)) per ciphertext
    for (u32 c = 0; c < count; c++) {
        if (he_status r = he_ct_automorph(c3 + (size_t)c * 3 * comp, ct_in + (size_t)c * 2 * comp, 1, 1, galois_elt,
                                          ctx, level, stream)) return r;
        HE_CUDA(cudaMemsetAsync(c3 + ((size_t)c * 3 + 1) * comp, 0, comp * 8, s));
        if (he_status r = he_ct_automorph(c3 + ((size_t)c * 3 + 2) * comp, ct_in + ((size_t)c * 2 + 1) * comp, 1, 1,
                                          galois_elt, ctx, level, stream)) return r;
    }
    return key_switch_common(ct_out, nullptr, nullptr, c3, count, galois_key, ctx, level, c3 + c3_words,
                             scratch_bytes - c3_words * 8, stream, false);
}

extern "C" he_status he_ct_matmul_tensor(uint64_t *t_out, const uint64_t *a, const uint64_t *b, uint32_t m,
                                         uint32_t k, uint32_t n, const he_context *ctx, uint32_t level,
                                         he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (he_status s = check_ptr(t_out, "t_out")) return s;
    if (he_status s = check_ptr(a, "a")) return s;
    if (he_status s = check_ptr(b, "b")) return s;
    if (m == 0 || k == 0 || n == 0) return fail(HE_EINVAL, "matrix dimensions must be positive");
    if ((u64)m * n * 3 * (level + 1) * ctx->N >= (1ull << 40)) return fail(HE_EINVAL, "matrix product too large");
    const u32 limbs = level + 1;
    const u64 threads = (u64)m * ((n + he::MM_TJ - 1) / he::MM_TJ) * limbs * (ctx->N / 2);
    he::k_ct_matmul_tensor<<<stream_grid(threads, 256), 256, 0, (cudaStream_t)stream>>>(
        t_out, a, b, m, k, n, (u32)ctx->log_n, limbs, ctx->tables->d_pc);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// ------------------------------------------------------------- encoding

struct he_encoder {
    const he_context *ctx = nullptr;
    u32 log_n = 0;                  // FFT length n = N / 2
    double2 *d_omega = nullptr;     // exp(-2 pi i j / n)
    double2 *d_zeta = nullptr;      // exp(i pi k / N), k < n
    u32 *d_slot = nullptr;          // slot of FFT index t
    u64 *d_primes = nullptr;        // (q_i, floor(2^64 / q_i)), i < n_data
    u64 *d_crt = nullptr;           // per-level CRT tables
    std::vector<size_t> crt_off;    // word offset of level l's table
    std::vector<u32> crt_nw;        // words per integer at level l
};

// Little-endian multi-word integers for the host-side CRT tables.
static void mw_mul_small(std::vector<u64> &a, u64 m)
{
    u64 carry = 0;
    for (u64 &w : a) {
        const u128 t = (u128)w * m + carry;
        w = (u64)t;
        carry = (u64)(t >> 64);
    }
    if (carry) a.push_back(carry);
}

static int mw_bits(const std::vector<u64> &a)
{
    for (size_t i = a.size(); i-- > 0;)
        if (a[i]) return (int)(64 * i) + bit_length(a[i]);
    return 0;
}

static void encoder_free(he_encoder *e)
{
    cudaFree(e->d_omega);
    cudaFree(e->d_zeta);
    cudaFree(e->d_slot);
    cudaFree(e->d_primes);
    cudaFree(e->d_crt);
    delete e;
}

extern "C" he_status he_encoder_create(const he_context *ctx, he_encoder **out)
{
    if (!out) return fail(HE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx) return fail(HE_EINVAL, "context is NULL");
    const u32 N = ctx->N, n = N / 2;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double2> omega(n), zeta(n);
    for (u32 j = 0; j < n; j++) {
        const long double a = 2 * pi * (long double)j / (long double)n;
        omega[j] = make_double2((double)cosl(a), (double)-sinl(a));
        const long double b = pi * (long double)j / (long double)N;
        zeta[j] = make_double2((double)cosl(b), (double)sinl(b));
    }
    std::vector<u32> slot(n);
    u64 e5 = 1;
    for (u32 j = 0; j < n; j++) {   // 5^j mod 2N = 4 t + 1
        slot[(e5 - 1) / 4] = j;
        e5 = e5 * 5 % (2 * (u64)N);
    }
    std::vector<u64> primes(2 * (size_t)ctx->n_data);
    for (u32 i = 0; i < ctx->n_data; i++) {
        primes[2 * i] = ctx->data[i];
        primes[2 * i + 1] = shoup(1, ctx->data[i]);
    }
    // CRT tables per level l (limbs q_0..q_l): Q, (Q - 1) / 2, Q / q_i,
    // then {q_i, (Q / q_i)^-1 mod q_i, its Shoup quotient}, then
    // 1 / (Q / 2^(64 (nw - 2))) for the estimate of the multiple of Q
    he_encoder *e = new he_encoder;
    e->ctx = ctx;
    e->log_n = (u32)(ctx->log_n - 1);
    std::vector<u64> crt;
    for (u32 l = 0; l < ctx->n_data; l++) {
        const u32 limbs = l + 1;
        std::vector<u64> Q{1};
        for (u32 i = 0; i < limbs; i++) mw_mul_small(Q, ctx->data[i]);
        const u32 nw = he::crt_words((u32)((mw_bits(Q) + 6 + 63) / 64));
        if (!nw) {
            delete e;
            return fail(HE_EUNSUPPORTED, "modulus chain too long for the CRT lift (level %u)", l);
        }
        e->crt_off.push_back(crt.size());
        e->crt_nw.push_back(nw);
        auto put = [&](const std::vector<u64> &x) {
            for (u32 w = 0; w < nw; w++) crt.push_back(w < x.size() ? x[w] : 0);
        };
        put(Q);
        std::vector<u64> Qh(Q);
        for (size_t w = 0; w < Qh.size(); w++) Qh[w] = (Qh[w] >> 1) | (w + 1 < Qh.size() ? Qh[w + 1] << 63 : 0);
        put(Qh);
        for (u32 i = 0; i < limbs; i++) {
            std::vector<u64> Qi{1};
            for (u32 j = 0; j < limbs; j++)
                if (j != i) mw_mul_small(Qi, ctx->data[j]);
            put(Qi);
        }
        for (u32 i = 0; i < limbs; i++) {
            const u64 q = ctx->data[i];
            u64 r = 1;
            for (u32 j = 0; j < limbs; j++)
                if (j != i) r = h_mul(r, ctx->data[j] % q, q);
            const u64 inv = h_inv(r, q);
            crt.insert(crt.end(), {q, inv, shoup(inv, q)});
        }
        // 1 / (Q / 2^(64 (nw - 2))), the reciprocal of the top two words
        std::vector<u64> Qp(Q);
        Qp.resize(nw, 0);
        const double qtop = std::ldexp((double)Qp[nw - 1], 64) + (double)Qp[nw - 2];
        const double inv = 1.0 / qtop;
        u64 bits;
        memcpy(&bits, &inv, 8);
        crt.push_back(bits);
    }
    cudaError_t ce = cudaSuccess;
    auto up = [&](auto **dst, const auto &src) {
        if (ce != cudaSuccess) return;
        const size_t bytes = src.size() * sizeof(src[0]);
        ce = cudaMalloc(dst, bytes);
        if (ce == cudaSuccess) ce = cudaMemcpy(*dst, src.data(), bytes, cudaMemcpyHostToDevice);
    };
    up(&e->d_omega, omega);
    up(&e->d_zeta, zeta);
    up(&e->d_slot, slot);
    up(&e->d_primes, primes);
    up(&e->d_crt, crt);
    if (ce != cudaSuccess) {
        encoder_free(e);
        return cuda_fail(ce, "encoder tables");
    }
    *out = e;
    return HE_OK;
}

extern "C" he_status he_encoder_destroy(he_encoder *enc)
{
    if (!enc) return HE_OK;   // like every *_destroy: NULL is a no-op
    encoder_free(enc);
    return HE_OK;
}

extern "C" size_t he_encode_scratch_bytes(const he_encoder *enc, uint32_t count)
{
    return enc ? (size_t)count * enc->ctx->N * 8 : 0;
}

extern "C" size_t he_decode_scratch_bytes(const he_encoder *enc, uint32_t level, uint32_t count)
{
    return enc ? (size_t)count * (level + 3) * enc->ctx->N * 8 : 0;
}

static he_status check_encode_args(const he_encoder *enc, uint32_t level, double scale)
{
    if (!enc) return fail(HE_EINVAL, "encoder is NULL");
    if (he_status s = check_level(enc->ctx, level, false)) return s;
    if (!(scale > 0) || !std::isfinite(scale)) return fail(HE_EINVAL, "scale must be finite and positive");
    return HE_OK;
}

static he::FftArgs fft_args(const he_encoder *enc, u32 count, u32 limbs, double scale)
{
    he::FftArgs a = {};
    a.omega = enc->d_omega;
    a.zeta = enc->d_zeta;
    a.slot_of = enc->d_slot;
    a.primes = enc->d_primes;
    a.scale = scale;
    a.inv_n = 1.0 / (double)(1u << enc->log_n);
    a.log_n = enc->log_n;
    a.log_n1 = enc->log_n / 2;
    a.limbs = limbs;
    a.count = count;
    return a;
}

extern "C" he_status he_encode(const he_encoder *enc, uint64_t *pt_out, const double *slots, uint32_t count,
                               double scale, uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_encode_args(enc, level, scale)) return s;
    if (he_status s = check_ptr(pt_out, "pt_out")) return s;
    if (he_status s = check_ptr(slots, "slots")) return s;
    if (count == 0) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < he_encode_scratch_bytes(enc, count)) return fail(HE_EINVAL, "scratch too small");
    if ((u64)count * (level + 1) * enc->ctx->N >= (1ull << 40)) return fail(HE_EINVAL, "batch too large");
    he::FftArgs a = fft_args(enc, count, level + 1, scale);
    a.z_in = (const double2 *)slots;
    a.pt_out = pt_out;
    a.u = (double2 *)scratch;
    HE_CUDA(he::launch_encode_fft(a, (cudaStream_t)stream));
    return ntt_launch(uniform_launch(pt_out, level + 1, count, enc->ctx->tables), enc->ctx->log_n, false,
                      (cudaStream_t)stream);
}

static he_status crt_compose(const he_encoder *enc, double *out, const uint64_t *coeffs, uint32_t count, uint32_t level,
                             cudaStream_t s)
{
    const u64 total = (u64)count * enc->ctx->N;
    HE_CUDA(he::launch_crt_compose(out, coeffs, enc->d_crt + enc->crt_off[level], enc->crt_nw[level],
                                   (u32)enc->ctx->log_n, level + 1, total, stream_grid(total, 128), s));
    return HE_OK;
}

extern "C" he_status he_crt_compose(const he_encoder *enc, double *out, const uint64_t *coeffs, uint32_t count,
                                    uint32_t level, he_stream_t stream)
{
    if (!enc) return fail(HE_EINVAL, "encoder is NULL");
    if (he_status s = check_level(enc->ctx, level, false)) return s;
    if (!out || ((uintptr_t)out & 7)) return fail(HE_EINVAL, "out is NULL or not 8-byte aligned");
    if (he_status s = check_ptr(coeffs, "coeffs")) return s;
    if (count == 0) return HE_OK;
    return crt_compose(enc, out, coeffs, count, level, (cudaStream_t)stream);
}

extern "C" he_status he_decode(const he_encoder *enc, double *slots_out, const uint64_t *pt, uint32_t count,
                               double scale, uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_encode_args(enc, level, scale)) return s;
    if (he_status s = check_ptr(slots_out, "slots_out")) return s;
    if (he_status s = check_ptr(pt, "pt")) return s;
    if (count == 0) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < he_decode_scratch_bytes(enc, level, count)) return fail(HE_EINVAL, "scratch too small");
    if ((u64)count * (level + 1) * enc->ctx->N >= (1ull << 40)) return fail(HE_EINVAL, "batch too large");
    const he_context *ctx = enc->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t words = (size_t)count * (level + 1) * ctx->N;
    u64 *coef = (u64 *)scratch;                            // [count][level + 1][N]
    double *m = (double *)(coef + words);                  // [count][N]
    double2 *u = (double2 *)(m + (size_t)count * ctx->N);  // [count][N / 2]
    HE_CUDA(cudaMemcpyAsync(coef, pt, words * 8, cudaMemcpyDeviceToDevice, s));
    if (he_status r = ntt_launch(uniform_launch(coef, level + 1, count, ctx->tables), ctx->log_n, true, s)) return r;
    if (he_status r = crt_compose(enc, m, coef, count, level, s)) return r;
    he::FftArgs a = fft_args(enc, count, level + 1, 1.0 / scale);
    a.m_in = m;
    a.z_out = (double2 *)slots_out;
    a.u = u;
    HE_CUDA(he::launch_decode_fft(a, s));
    return HE_OK;
}

// ------------------------------------------------------------- encryption

extern "C" size_t he_encrypt_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count)
{
    return ctx ? (size_t)count * 3 * (level + 1) * ctx->N * 8 : 0;
}

// Encryption with the draws given (v non-NULL) or generated from `seed`.
static he_status encrypt_common(uint64_t *ct_out, const uint64_t *pt, const uint64_t *pk, const int8_t *v,
                                const int8_t *e0, const int8_t *e1, uint64_t seed, uint32_t count,
                                const he_context *ctx, uint32_t level, void *scratch, size_t scratch_bytes,
                                he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, false)) return s;
    if (he_status s = check_ptr(ct_out, "ct_out")) return s;
    if (he_status s = check_ptr(pt, "pt")) return s;
    if (he_status s = check_ptr(pk, "pk")) return s;
    if (count == 0) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < he_encrypt_scratch_bytes(ctx, level, count)) return fail(HE_EINVAL, "scratch too small");
    if ((u64)count * 3 * (level + 1) * (ctx->N / 4096 + 1) > 0x7fffffffull) return fail(HE_EINVAL, "batch too large");
    const u32 n = level + 1;
    cudaStream_t s = (cudaStream_t)stream;
    u64 *noise = (u64 *)scratch;
    const u64 words = (u64)count * 3 * n * ctx->N;
    if (v)
        he::k_enc_noise<<<stream_grid(words, 256), 256, 0, s>>>(noise, v, e0, e1, (u32)ctx->log_n, n, count,
                                                                 ctx->tables->d_pc);
    else
        he::k_enc_noise_seeded<<<stream_grid(words, 256), 256, 0, s>>>(noise, seed, (u32)ctx->log_n, n, count,
                                                                        ctx->tables->d_pc);
    HE_CUDA(cudaGetLastError());
    if (he_status r = ntt_launch(uniform_launch(noise, n, 3 * count, ctx->tables), ctx->log_n, false, s)) return r;
    he::k_enc_combine<<<stream_grid((u64)count * n * ctx->N, 256), 256, 0, s>>>(
        ct_out, noise, pt, pk, (u32)ctx->log_n, n, count, ctx->n_data, ctx->tables->d_pc);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

extern "C" he_status he_encrypt(uint64_t *ct_out, const uint64_t *pt, const uint64_t *pk, const int8_t *v,
                                const int8_t *e0, const int8_t *e1, uint32_t count, const he_context *ctx,
                                uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream)
{
    if (!v || !e0 || !e1) return fail(HE_EINVAL, "v, e0 or e1 is NULL");
    return encrypt_common(ct_out, pt, pk, v, e0, e1, 0, count, ctx, level, scratch, scratch_bytes, stream);
}

extern "C" he_status he_encrypt_seeded(uint64_t *ct_out, const uint64_t *pt, const uint64_t *pk, uint64_t seed,
                                       uint32_t count, const he_context *ctx, uint32_t level, void *scratch,
                                       size_t scratch_bytes, he_stream_t stream)
{
    return encrypt_common(ct_out, pt, pk, nullptr, nullptr, nullptr, seed, count, ctx, level, scratch, scratch_bytes,
                          stream);
}

extern "C" he_status he_sample_encryption_draws(int8_t *v, int8_t *e0, int8_t *e1, uint32_t count, uint32_t N,
                                                uint64_t seed, he_stream_t stream)
{
    int log_n;
    if (he_status s = check_degree(N, &log_n)) return s;
    if (!v || !e0 || !e1) return fail(HE_EINVAL, "v, e0 or e1 is NULL");
    if (count == 0) return HE_OK;
    if ((u64)count * N > (1ull << 40)) return fail(HE_EINVAL, "batch too large");
    he::k_enc_draws<<<stream_grid((u64)count * N, 256), 256, 0, (cudaStream_t)stream>>>(v, e0, e1, seed,
                                                                                        (u32)log_n, count);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// ------------------------------------------------------------- measurement

// Register-resident butterfly probe: each thread runs `iters` rounds of 8
// independent Harvey butterflies (Algorithm 1) on a 60-bit prime with no
// memory traffic, so the launch measures the integer-pipe ceiling of the
// transform's arithmetic. One word per thread is written so nothing is
// optimised away.
__global__ void k_butterfly_probe(u64 *sink, const he::PrimeConst c, u64 w, u64 w_sh, u32 iters)
{
    const u64 p = c.p;
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = (threadIdx.x * 977 + blockIdx.x * 131 + i * 7919) % p;
    for (u32 it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) he::ct_butterfly(x[i], x[i + 8], w, w_sh, c);
#pragma unroll
        for (int i = 0; i < 8; i++) he::ct_butterfly(x[2 * (i & 3) + (i >> 2) * 8], x[2 * (i & 3) + 1 + (i >> 2) * 8],
                                                     w, w_sh, c);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

extern "C" he_status he_butterfly_probe(uint64_t *sink, uint32_t blocks, uint32_t threads, uint32_t iters,
                                        he_stream_t stream)
{
    if (he_status s = check_ptr(sink, "sink")) return s;
    if (!blocks || !threads || threads > 1024 || (threads & 31)) return fail(HE_EINVAL, "bad probe shape");
    const u64 p = 1152921504606584833ull;   // the largest 60-bit prime = 1 mod 2^16
    const u64 w = 123456789012345ull % p;
    k_butterfly_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(sink, prime_const(p, 1u << 15, w), w,
                                                                    shoup(w, p), iters);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// FP64 throughput probe: each thread runs 8 independent chains of `iters`
// fused multiply-adds (x <- x a + b) in registers, 16 FLOP per step, and
// writes one double. Timing the launch gives the FP64 rate that bounds the
// slot FFT of encoding and decoding.
__global__ void k_fp64_probe(double *sink, u32 iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (u32 it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
    }
    double acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc += x[i];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

extern "C" he_status he_fp64_probe(double *sink, uint32_t blocks, uint32_t threads, uint32_t iters, he_stream_t stream)
{
    if (!sink || ((uintptr_t)sink & 7)) return fail(HE_EINVAL, "sink is NULL or not 8-byte aligned");
    if (!blocks || !threads || threads > 1024 || (threads & 31)) return fail(HE_EINVAL, "bad probe shape");
    k_fp64_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(sink, iters, 0.999999, 1e-7);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// Elementwise application of the transform butterflies, so that their
// contract can be checked on the device: forward (Algorithm 1 with the range
// [0, 8p + 2^32)) or inverse (Gentleman-Sande on [0, 4p)).
__global__ void k_butterfly_apply(u64 *x, u64 *y, const u64 *w, const u64 *w_sh, u32 n, const he::PrimeConst c,
                                  int inverse)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u64 a = x[i], b = y[i];
    if (inverse)
        he::gs_butterfly(a, b, w[i], w_sh[i], c);
    else
        he::ct_butterfly(a, b, w[i], w_sh[i], c);
    x[i] = a;
    y[i] = b;
}

extern "C" he_status he_butterfly_apply(uint64_t *x, uint64_t *y, const uint64_t *w, const uint64_t *w_shoup,
                                        uint32_t n, uint64_t p, int32_t inverse, he_stream_t stream)
{
    if (he_status s = check_modulus_range(p)) return s;
    if (!n) return HE_OK;
    if (!x || !y || !w || !w_shoup) return fail(HE_EINVAL, "NULL array");
    k_butterfly_apply<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, y, w, w_shoup, n,
                                                                       prime_const(p, 1024, 1), inverse);
    HE_CUDA(cudaGetLastError());
    return HE_OK;
}

// ------------------------------------------------------------------- plans

struct he_plan {
    struct Group {
        int log_n;
        int log_b;
        int log_e;
        u32 items;
        u32 clusters;                  // persistent grid (0: one cluster per limb)
        he::LimbJob *d_jobs;
    };
    std::vector<Group> groups;         // per-degree launches
    bool mixed = false;                // one mixed-degree launch per direction
    he::MixedUnit *d_units = nullptr;
    he::LimbJob *d_mixed_jobs = nullptr;
    u32 n_units = 0;
    u32 clusters_fwd = 0, clusters_inv = 0;
};

extern "C" he_status he_plan_destroy(he_plan *plan)
{
    if (plan) {
        cudaDeviceSynchronize();
        for (auto &g : plan->groups) cudaFree(g.d_jobs);
        cudaFree(plan->d_units);
        cudaFree(plan->d_mixed_jobs);
        delete plan;
    }
    return HE_OK;
}

template <class T>
static cudaError_t upload(T **dst, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

extern "C" he_status he_ntt_plan_create(const he_poly_desc *descs_host, uint32_t count,
                                        const he_ntt_shape *shapes_host, uint32_t n_shapes, he_plan **out)
{
    if (!out) return fail(HE_EINVAL, "out is NULL");
    *out = nullptr;
    if (count && !descs_host) return fail(HE_EINVAL, "descs_host is NULL");
    if (n_shapes && !shapes_host) return fail(HE_EINVAL, "shapes_host is NULL");
    std::map<int, std::vector<he::LimbJob>> by_degree;
    for (u32 i = 0; i < count; i++) {
        const he_poly_desc &d = descs_host[i];
        int log_n;
        if (!d.tables) return fail(HE_EINVAL, "descriptor %u has no tables", i);
        if (he_status s = check_degree(d.N, &log_n)) return s;
        if (d.tables->N != d.N) return fail(HE_EINVAL, "descriptor %u: tables are for N = %u", i, d.tables->N);
        if ((u64)d.first_prime + d.limbs > d.tables->K)
            return fail(HE_EINVAL, "descriptor %u: primes %u..%u beyond the tables' %u", i, d.first_prime,
                        d.first_prime + d.limbs, d.tables->K);
        if (d.limbs && (!d.data || ((uintptr_t)d.data & 31)))
            return fail(HE_EINVAL, "descriptor %u: data NULL or not 32-byte aligned", i);
        for (u32 l = 0; l < d.limbs; l++) {
            he::LimbJob j;
            const u32 pr = d.first_prime + l;
            j.data = d.data + (size_t)l * d.N;
            j.tw_fwd = d.tables->d_fwd + (size_t)pr * d.N;
            j.tw_inv = d.tables->d_inv + (size_t)pr * d.N;
            j.pc = d.tables->d_pc + pr;
            by_degree[log_n].push_back(j);
        }
    }
    for (u32 s = 0; s < n_shapes; s++) {
        int log_n;
        if (he_status st = check_degree(shapes_host[s].N, &log_n)) return st;
        const he::DegreeOps *ops = he::degree_ops(log_n);
        if (shapes_host[s].log_thread_words > 15 || shapes_host[s].ctas_per_sm > 32)
            return fail(HE_EINVAL, "shape %u: log_thread_words or ctas_per_sm out of range", s);
        if (!ops->has_shape((int)shapes_host[s].log_block,
                            thread_words_code(shapes_host[s].log_thread_words, shapes_host[s].ctas_per_sm)))
            return fail(HE_EUNSUPPORTED,
                        "no kernel with 2^%u words per CTA, 2^%u per thread and %u CTAs per SM for N = 2^%d",
                        shapes_host[s].log_block, shapes_host[s].log_thread_words, shapes_host[s].ctas_per_sm, log_n);
    }
    he_plan *plan = new he_plan;
    bool mixed = n_shapes == 0 && !by_degree.empty();
    for (auto &kv : by_degree) mixed = mixed && kv.first >= 12 && kv.first <= 15;
    if (mixed) {
        // largest degrees first, so that the long units start early
        std::vector<he::LimbJob> jobs;
        std::vector<he::MixedUnit> units;
        for (auto it = by_degree.rbegin(); it != by_degree.rend(); ++it) {
            const u32 per = 8u >> (it->first - 12);
            for (size_t k = 0; k < it->second.size(); k += per) {
                he::MixedUnit u;
                u.log_n = (u32)it->first;
                u.first_job = (u32)jobs.size();
                u.n_jobs = (u32)std::min<size_t>(per, it->second.size() - k);
                u.pad = 0;
                for (u32 q = 0; q < u.n_jobs; q++) jobs.push_back(it->second[k + q]);
                units.push_back(u);
            }
        }
        cudaError_t e = upload(&plan->d_mixed_jobs, jobs);
        if (e == cudaSuccess) e = upload(&plan->d_units, units);
        if (e != cudaSuccess) {
            he_plan_destroy(plan);
            return cuda_fail(e, "plan work list");
        }
        plan->mixed = true;
        plan->n_units = (u32)units.size();
        // one cluster per unit: measured faster than a persistent grid of
        // co-resident clusters walking the units (independent clusters keep
        // every SM busy with CTAs in different phases)
        plan->clusters_fwd = plan->n_units;
        plan->clusters_inv = plan->n_units;
        *out = plan;
        return HE_OK;
    }
    for (auto &kv : by_degree) {
        he_plan::Group g = {};
        g.log_n = kv.first;
        const he::DegreeOps *ops = he::degree_ops(g.log_n);
        g.log_b = ops->default_log_b;
        g.log_e = ops->default_log_e;
        bool persistent = false;
        for (u32 s = 0; s < n_shapes; s++)
            if (shapes_host[s].N == (1u << g.log_n) && shapes_host[s].log_block) {
                g.log_b = (int)shapes_host[s].log_block;
                g.log_e = thread_words_code(shapes_host[s].log_thread_words ? shapes_host[s].log_thread_words : 4,
                                            shapes_host[s].ctas_per_sm);
                persistent = shapes_host[s].persistent != 0;
            }
        g.items = (u32)kv.second.size();
        if (persistent) {
            const int mc = std::max(ops->max_clusters(g.log_b, g.log_e, false), 1);
            g.clusters = std::min<u32>(g.items, (u32)mc);
        }
        cudaError_t e = upload(&g.d_jobs, kv.second);
        if (e != cudaSuccess) {
            he_plan_destroy(plan);
            return cuda_fail(e, "plan job list");
        }
        plan->groups.push_back(g);
    }
    *out = plan;
    return HE_OK;
}

static he_status plan_run(const he_plan *plan, he_stream_t stream, bool inv)
{
    if (!plan) return fail(HE_EINVAL, "plan is NULL");
    if (plan->mixed) {
        HE_CUDA(he::launch_ntt_mixed(plan->d_units, plan->n_units, plan->d_mixed_jobs, inv,
                                     inv ? plan->clusters_inv : plan->clusters_fwd, (cudaStream_t)stream));
        return HE_OK;
    }
    for (const auto &g : plan->groups) {
        he::NttLaunch a = {};
        a.items = g.items;
        a.jobs = g.d_jobs;
        if (g.clusters)
            HE_CUDA(he::degree_ops(g.log_n)->ntt_persistent(a, g.log_b, g.log_e, inv, g.clusters,
                                                            (cudaStream_t)stream));
        else
            HE_CUDA(he::degree_ops(g.log_n)->ntt(a, g.log_b, g.log_e, inv, (cudaStream_t)stream));
    }
    return HE_OK;
}

extern "C" he_status he_ntt_plan_fwd(const he_plan *plan, he_stream_t stream) { return plan_run(plan, stream, false); }
extern "C" he_status he_ntt_plan_inv(const he_plan *plan, he_stream_t stream) { return plan_run(plan, stream, true); }

extern "C" uint32_t he_plan_launches(const he_plan *plan)
{
    return plan ? (plan->mixed ? 1u : (uint32_t)plan->groups.size()) : 0;
}

// ------------------------------------------------ host-resident batches
//
// The asynchronous pipeline of Sec. III for data that lives in host memory:
// chunk c of the batch goes to internal stream c mod S and scratch slot
// c mod S, where it is copied in, transformed and copied out. Chunks on one
// stream run in order, so a slot is reused only after its previous chunk has
// been copied out; chunks on different streams overlap, which lets the two
// copy directions and the kernels run at the same time. The caller's stream
// forks into the internal streams with one event and joins them with one
// event per stream, so the call is ordered like any other stream operation
// and stays capturable. Streams and events are created once per device and
// reused; the mutex keeps concurrent callers from interleaving their event
// records.
static const int kHostStreams = 4;
static const u32 kHostMinChunks = 16;   // chunks per batch when the scratch allows

struct HostPipeline {
    std::mutex mu;
    bool ready = false;
    cudaStream_t st[kHostStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kHostStreams] = {};
};

static std::mutex g_host_pipeline_init;
static HostPipeline g_host_pipeline[256];   // per device ordinal

static he_status host_pipeline(HostPipeline **out)
{
    int dev = 0;
    HE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(HE_EUNSUPPORTED, "device ordinal %d out of range", dev);
    HostPipeline &p = g_host_pipeline[dev];
    std::lock_guard<std::mutex> lock(g_host_pipeline_init);
    if (!p.ready) {
        HE_CUDA(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
        for (int i = 0; i < kHostStreams; i++) {
            HE_CUDA(cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking));
            HE_CUDA(cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming));
        }
        p.ready = true;
    }
    *out = &p;
    return HE_OK;
}

extern "C" he_status he_ntt_host(const uint64_t *in_host, uint64_t *out_host, uint32_t N, uint32_t limbs,
                                 uint32_t count, const uint64_t *moduli_host, const he_ntt_tables *tw, uint32_t ops,
                                 uint64_t *work, size_t work_bytes, he_stream_t stream)
{
    int log_n;
    if (he_status s = check_poly_args(work, N, limbs, moduli_host, tw, &log_n)) return s;
    if (ops == 0 || (ops & ~(HE_NTT_OP_FORWARD | HE_NTT_OP_INVERSE)))
        return fail(HE_EINVAL, "ops must be HE_NTT_OP_FORWARD, HE_NTT_OP_INVERSE or both, got %u", ops);
    if ((u64)limbs * count == 0) return HE_OK;
    if (!in_host || !out_host) return fail(HE_EINVAL, "host buffer is NULL");
    const size_t poly_words = (size_t)limbs * N;
    const size_t poly_bytes = poly_words * 8;
    const size_t total_bytes = poly_bytes * count;
    const uintptr_t ib = (uintptr_t)in_host, ob = (uintptr_t)out_host;
    if (ib != ob && ib < ob + total_bytes && ob < ib + total_bytes)
        return fail(HE_EINVAL, "in_host and out_host overlap without being equal");
    const size_t fit = work_bytes / poly_bytes;
    if (fit == 0)
        return fail(HE_EINVAL, "scratch of %zu bytes holds no polynomial of %zu bytes", work_bytes, poly_bytes);
    const u32 slots = (u32)std::min<size_t>({(size_t)kHostStreams, fit, (size_t)count});
    const u32 want = (count + kHostMinChunks - 1) / kHostMinChunks;
    const u32 chunk = (u32)std::max<size_t>(1, std::min<size_t>(fit / slots, want));
    const u32 chunks = (count + chunk - 1) / chunk;
    const bool fwd = ops & HE_NTT_OP_FORWARD, inv = ops & HE_NTT_OP_INVERSE;

    HostPipeline *p = nullptr;
    if (he_status s = host_pipeline(&p)) return s;
    std::lock_guard<std::mutex> lock(p->mu);
    cudaStream_t caller = (cudaStream_t)stream;
    HE_CUDA(cudaEventRecord(p->fork, caller));
    const u32 used = std::min(slots, chunks);
    for (u32 i = 0; i < used; i++) HE_CUDA(cudaStreamWaitEvent(p->st[i], p->fork, 0));

    he_status status = HE_OK;
    for (u32 c = 0; c < chunks && status == HE_OK; c++) {
        const u32 i = c % slots;
        const u32 n = std::min(chunk, count - c * chunk);
        const size_t off = (size_t)c * chunk * poly_words;
        uint64_t *dev = work + (size_t)i * chunk * poly_words;
        cudaError_t e = cudaMemcpyAsync(dev, in_host + off, n * poly_bytes, cudaMemcpyHostToDevice, p->st[i]);
        if (e != cudaSuccess) {
            status = cuda_fail(e, "copy to device");
            break;
        }
        if (fwd) status = ntt_common(dev, N, limbs, n, moduli_host, tw, (he_stream_t)p->st[i], false);
        if (status == HE_OK && inv) status = ntt_common(dev, N, limbs, n, moduli_host, tw, (he_stream_t)p->st[i], true);
        if (status != HE_OK) break;
        e = cudaMemcpyAsync(out_host + off, dev, n * poly_bytes, cudaMemcpyDeviceToHost, p->st[i]);
        if (e != cudaSuccess) status = cuda_fail(e, "copy to host");
    }
    // join even after a failure, so that the caller's stream stays ordered
    // after whatever was queued
    for (u32 i = 0; i < used; i++) {
        cudaError_t e = cudaEventRecord(p->join[i], p->st[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, p->join[i], 0);
        if (e != cudaSuccess && status == HE_OK) status = cuda_fail(e, "join the pipeline streams");
    }
    return status;
}

// ---- multi-degree MulLinRS batches (one launch per pipeline stage) -------

static he_status check_multi_jobs(const he_mrr_multi_job *jobs, uint32_t n_jobs, bool pointers)
{
    if (n_jobs && !jobs) return fail(HE_EINVAL, "jobs_host is NULL");
    for (u32 i = 0; i < n_jobs; i++) {
        const he_mrr_multi_job &J = jobs[i];
        if (!J.ctx) return fail(HE_EINVAL, "job %u: context is NULL", i);
        if (J.ctx->log_n < 12 || J.ctx->log_n > 15)
            return fail(HE_EUNSUPPORTED, "job %u: degree %u outside [2^12, 2^15]", i, J.ctx->N);
        if (he_status s = check_level(J.ctx, J.level, true)) return s;
        if (J.count > 4096) return fail(HE_EINVAL, "job %u: more than 4096 ciphertext pairs", i);
        if (!J.count || !pointers) continue;
        if (!J.key || J.key->ctx != J.ctx) return fail(HE_EINVAL, "job %u: key is NULL or of another context", i);
        if (he_status s = check_ptr(J.ct_out, "ct_out")) return s;
        if (he_status s = check_ptr(J.ct_a, "ct_a")) return s;
        if (he_status s = check_ptr(J.ct_b, "ct_b")) return s;
    }
    return HE_OK;
}

extern "C" size_t he_mul_relin_rescale_multi_scratch_bytes(const he_mrr_multi_job *jobs_host, uint32_t n_jobs)
{
    if (check_multi_jobs(jobs_host, n_jobs, false) != HE_OK) return 0;
    size_t words = 0;
    for (u32 i = 0; i < n_jobs; i++) words += mrr_job_words(jobs_host[i].ctx, jobs_host[i].level + 1, jobs_host[i].count);
    return words * 8;
}

// One pass over up to kMaxJobs jobs whose scratch starts at w. Per job:
// c2 [count][n][N], accq [count][2][n][N], lift2 [count][2][N], the
// expanded mod-up buffer [count][n + 1][n][N], plift [count][2][N].
static he_status mrr_multi_pass(const he_mrr_multi_job *jobs, u32 n_jobs, u64 *w, cudaStream_t s)
{
    he::JobTable t = {};
    u64 tot[he::JS_COUNT] = {};
    for (u32 i = 0; i < n_jobs; i++) {
        const he_mrr_multi_job &J = jobs[i];
        const he_context *ctx = J.ctx;
        const u32 n = J.level + 1, c = J.count;
        const size_t N = ctx->N;
        he::EvalJob &E = t.job[t.n_jobs++];
        E.ct_a = J.ct_a;
        E.ct_b = J.ct_b;
        E.out = J.ct_out;
        E.n = n;
        E.count = c;
        E.evk = J.key->d_evk;
        E.ctx = dev_ctx(ctx);
        E.c2 = w;
        E.accq = E.c2 + (size_t)c * n * N;
        E.lift2 = E.accq + (size_t)c * 2 * n * N;
        E.mx = E.lift2 + (size_t)c * 2 * N;
        E.plift = E.mx + (size_t)c * (n + 1) * n * N;
        w = E.plift + (size_t)c * 2 * N;
        const u64 per = 8u >> (ctx->log_n - 12);     // items side by side in one cluster
        auto units = [&](u64 items) { return (items + per - 1) / per; };
        u64 cnt[he::JS_COUNT] = {};
        cnt[he::JS_DIGITS] = units((u64)c * n);
        cnt[he::JS_EXPAND] = units((u64)c * n * n);
        cnt[he::JS_MAC] = (u64)(c + he::MAC_CTS - 1) / he::MAC_CTS * (n + 1) * (N / 2);
        cnt[he::JS_LAST] = units(2ull * c);
        cnt[he::JS_REST] = units(2ull * c * (n - 1));
        cnt[he::JS_PLIFT] = units(2ull * c);
        for (int st = 0; st < he::JS_COUNT; st++) {
            if (tot[st] + cnt[st] > 0x0fffffffull) return fail(HE_EINVAL, "batch too large");
            E.begin[st] = (u32)tot[st];
            tot[st] += cnt[st];
        }
    }
    he::EvalArgs a = {};
    a.evk = t.job[0].evk;   // every stage binds its job's own context and key
    a.ctx = t.job[0].ctx;
    a.n = t.job[0].n;
    HE_CUDA(he::launch_mrr_multi(he::MS_DIGITS, a, t, (u32)tot[he::JS_DIGITS], s));
    HE_CUDA(he::launch_mrr_multi(he::MS_EXPAND, a, t, (u32)tot[he::JS_EXPAND], s));
    he::k_ks_mac<true><<<stream_grid(tot[he::JS_MAC], 256), 256, 0, s>>>(a, 0, (u32)tot[he::JS_MAC], t);
    HE_CUDA(cudaGetLastError());
    HE_CUDA(he::launch_mrr_multi(he::MS_PLIFT, a, t, (u32)tot[he::JS_PLIFT], s));
    HE_CUDA(he::launch_mrr_multi(he::MS_LAST, a, t, (u32)tot[he::JS_LAST], s));
    HE_CUDA(he::launch_mrr_multi(he::MS_REST_Z, a, t, (u32)tot[he::JS_REST], s));
    HE_CUDA(he::launch_mrr_multi(he::MS_REST_OUT, a, t, (u32)tot[he::JS_REST], s));
    return HE_OK;
}

extern "C" he_status he_mul_relin_rescale_multi(const he_mrr_multi_job *jobs_host, uint32_t n_jobs, void *scratch,
                                                size_t scratch_bytes, he_stream_t stream)
{
    if (he_status s = check_multi_jobs(jobs_host, n_jobs, true)) return s;
    std::vector<he_mrr_multi_job> live;
    for (u32 i = 0; i < n_jobs; i++)
        if (jobs_host[i].count) live.push_back(jobs_host[i]);
    if (live.empty()) return HE_OK;
    if (he_status s = check_ptr(scratch, "scratch")) return s;
    if (scratch_bytes < he_mul_relin_rescale_multi_scratch_bytes(live.data(), (u32)live.size()))
        return fail(HE_EINVAL, "scratch too small");
    u64 *w = (u64 *)scratch;
    for (size_t i = 0; i < live.size(); i += he::kMaxJobs) {
        const u32 m = (u32)std::min<size_t>(he::kMaxJobs, live.size() - i);
        if (he_status r = mrr_multi_pass(live.data() + i, m, w, (cudaStream_t)stream)) return r;
        for (u32 k = 0; k < m; k++) w += mrr_job_words(live[i + k].ctx, live[i + k].level + 1, live[i + k].count);
    }
    return HE_OK;
}

// ------------------------------------------- allocation-free MulLinRS
//
// Some callers cannot allocate device memory at the point where they need a
// mul-relin-rescale: code that runs while a stream is being captured (plain
// cudaMalloc is not allowed there), latency-critical serving paths that must
// never block on the device allocator (cudaMalloc can synchronise the whole
// device), and embedders whose device memory is owned and budgeted by another
// runtime. he_mul_relin_rescale_noalloc serves them: it runs the same kernels
// as he_mul_relin_rescale with the key-switching and rescale scratch taken
// from a fixed buffer compiled into this library, so the call itself never
// allocates.
//
// The buffer is a file-scope __device__ array of HE_NOALLOC_SCRATCH_BYTES;
// every GPU that loads the library holds it until the process exits. Host
// code cannot use the array's name as a device address, so the first call on
// each device resolves the address with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should therefore come
// before any stream capture. All calls share the one buffer: calls that may
// overlap on the GPU (different streams without ordering between them) race
// on it and must be serialised by the caller. Each kernel writes every
// scratch word it later reads within the same call, so nothing in the buffer
// needs to start at zero and the contents left by a previous call are
// harmless.
static const size_t kNoAllocScratchBytes = (size_t)HE_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchBytes / 8];

// The resolved address belongs to the device's current context: after a
// cudaDeviceReset (or any teardown and re-creation of the context) the module
// is loaded again and the array may sit elsewhere. So the cache is keyed by
// device ordinal AND the context's process-unique id (cuCtxGetId, fetched
// through the runtime's driver entry points, so the library needs no link
// against the driver library), and a changed id resolves the address again.
struct NoAllocSlot {
    unsigned long long ctx_id;   // 0: never resolved
    void *addr;
};
static std::mutex g_noalloc_mutex;
static NoAllocSlot g_noalloc_slot[256];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if there is none yet).
static he_status current_context_id(unsigned long long *id)
{
    static std::once_flag once;
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PfnCtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PfnCtxGetId)f;
    });
    if (!get_current || !get_id) return fail(HE_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return fail(HE_ECUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (c && get_id(c, id) != CUDA_SUCCESS) return fail(HE_ECUDA, "cuCtxGetId failed");
    return HE_OK;
}

static he_status noalloc_scratch_address(void **out)
{
    int dev = 0;
    HE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(HE_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    if (he_status s = current_context_id(&id)) return s;
    NoAllocSlot &slot = g_noalloc_slot[dev];
    if (id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // makes the device's context current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(built-in scratch)");
        if (he_status s = current_context_id(&id)) return s;
        if (id == 0) return fail(HE_ECUDA, "no current context after resolving the built-in scratch");
        slot.ctx_id = id;
        slot.addr = p;
    }
    *out = slot.addr;
    return HE_OK;
}

extern "C" he_status he_mul_relin_rescale_noalloc(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b,
                                                  uint32_t count, const he_relin_key *key, const he_context *ctx,
                                                  uint32_t level, he_stream_t stream)
{
    if (he_status s = check_level(ctx, level, true)) return s;
    if (count == 0) return HE_OK;
    const size_t need = mrr_words(ctx, level + 1) * 8 * (size_t)count;
    if (need > kNoAllocScratchBytes)
        return fail(HE_EINVAL,
                    "mul-relin-rescale of %u pair(s) at N = %u, level %u needs %zu bytes of scratch; the built-in "
                    "buffer holds %zu bytes (use he_mul_relin_rescale with caller scratch, or fewer pairs)",
                    count, ctx->N, level, need, kNoAllocScratchBytes);
    void *scratch = nullptr;
    if (he_status s = noalloc_scratch_address(&scratch)) return s;
    return he_mul_relin_rescale(ct_out, ct_a, ct_b, count, key, ctx, level, scratch, kNoAllocScratchBytes, stream);
}

// ------------------------------------------------------- degree dispatch

namespace he {
extern const DegreeOps degree_ops_10, degree_ops_11, degree_ops_12, degree_ops_13, degree_ops_14,
    degree_ops_15, degree_ops_16;

const DegreeOps *degree_ops(int log_n)
{
    switch (log_n) {
    case 10: return &degree_ops_10;
    case 11: return &degree_ops_11;
    case 12: return &degree_ops_12;
    case 13: return &degree_ops_13;
    case 14: return &degree_ops_14;
    case 15: return &degree_ops_15;
    case 16: return &degree_ops_16;
    default: return nullptr;
    }
}
}  // namespace he
