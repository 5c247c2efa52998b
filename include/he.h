/*
 * he.h -- C ABI of the GB300 CKKS hot-path library (libhe.so).
 *
 * The library implements the data-parallel evaluation path of CKKS as
 * described in "Accelerating Encrypted Computing on Intel GPUs" (arXiv
 * 2109.14704): the negacyclic NTT and inverse NTT over RNS limbs of 64-bit
 * words (Sec. II-B, Sec. III-B, Algorithm 1), the NTT-domain dyadic product
 * (Sec. II-B), and the evaluation routines Mul, Relin and RS (Sec. II-A),
 * plus batched plans that run many polynomials or ciphertexts in one launch
 * (Sec. III-B "parallelism of NTT for HE", Sec. III asynchronous pipeline).
 *
 * Conventions shared by every call
 * --------------------------------
 * Words.    Every coefficient is a uint64_t residue. Moduli are odd primes
 *           2^30 <= q < 2^60 with q = 1 mod 2N (Sec. III-A-1 bounds them below 60
 *           bits so that lazy reduction and the fused multiply-add never
 *           overflow a 64-bit word).
 * Layout.   Limb-major and contiguous: a polynomial with L limbs is
 *           poly[l * N + i]; a ciphertext with n limbs and c components is
 *           ct[(k * n + l) * N + i]. Device buffers must be 32-byte aligned
 *           (the transforms move runs of words with 256-bit accesses).
 * Domains.  Ciphertexts and keys are in the NTT domain, in the bit-reversed
 *           evaluation order of he_ntt_fwd.
 * Ranges.   Inputs must be canonical (in [0, q)); outputs are always
 *           canonical. Lazy ranges never cross this interface.
 * Memory.   Pointers named *_host are host memory; every other data pointer
 *           is device memory owned by the caller. The library owns only the
 *           opaque handles (tables, contexts, keys, plans, encoders), until
 *           *_destroy; a *_destroy of NULL does nothing and returns HE_OK.
 *           Scratch buffers are passed in by the caller; he_*_scratch_bytes
 *           gives their size.
 * Streams.  Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy
 *           default stream). Only *_create, *_upload and *_destroy
 *           synchronise; no other call blocks the host (Sec. III: the host
 *           synchronises only when results are read back).
 * Errors.   Every call returns an he_status, except he_version,
 *           he_plan_launches and the size queries (he_*_scratch_bytes, 0
 *           for bad arguments). Argument checks run on the host
 *           before anything is enqueued and return HE_EINVAL without side
 *           effects. A failed CUDA call returns HE_ECUDA; errors raised later
 *           by enqueued work surface at the caller's next synchronisation.
 *           he_last_error() gives a message for the calling thread's last
 *           failure.
 * Aliasing. Outputs must not overlap inputs unless a call says it works in
 *           place.
 */
#ifndef HE_H
#define HE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t he_status;
enum {
    HE_OK = 0,
    HE_EINVAL = -1,        /* bad argument (size, modulus, pointer, level) */
    HE_ENOMEM = -2,        /* device or host allocation failed             */
    HE_ECUDA = -3,         /* a CUDA runtime call failed                   */
    HE_EUNSUPPORTED = -4,  /* valid but not built (e.g. N outside 2^10..2^16) */
    HE_ETIMEOUT = -5       /* a bounded device-side wait gave up           */
};

typedef struct CUstream_st *he_stream_t;          /* same type as cudaStream_t */
typedef struct he_ntt_tables he_ntt_tables;       /* twiddles of K primes at one N */
typedef struct he_context he_context;             /* modulus chain q_0..q_L, P   */
typedef struct he_relin_key he_relin_key;         /* device copy of evk          */
typedef struct he_plan he_plan;                   /* a batched, replayable launch */

/* Message of the calling thread's last failed call ("" if none). Copies at
 * most len - 1 bytes and a terminating NUL into buf. */
he_status he_last_error(char *buf, size_t len);

/* Library version as 0xMMmmpp. */
uint32_t he_version(void);

/* ---- parameters ------------------------------------------------------------ */

/* The `count` largest primes q with exactly `bits` bits (2..60) and
 * q = 1 mod two_n, skipping the `n_exclude` values in exclude_host, written in
 * descending order to out_host. RNS moduli of Sec. II-B. Returns HE_EINVAL if
 * fewer than `count` exist. Host only. */
he_status he_primes_generate(uint32_t bits, uint64_t two_n, uint32_t count,
                             const uint64_t *exclude_host, uint32_t n_exclude,
                             uint64_t *out_host);

/* Twiddle tables for `limbs` primes at degree N (a power of two in
 * [2^10, 2^16]). For each prime q: psi = the smallest primitive 2N-th root of
 * unity mod q (Sec. II-B names psi; the smallest is this library's choice),
 * forward powers psi^brv(k) and inverse powers psi^-brv(k), k < N, each with
 * its Shoup quotient floor(W 2^64 / q) (the W' of Algorithm 1), and N^-1.
 * Synchronises. Device memory: 32 N bytes per prime. */
he_status he_ntt_tables_create(uint32_t N, uint32_t limbs, const uint64_t *moduli_host,
                               he_ntt_tables **out);
he_status he_ntt_tables_destroy(he_ntt_tables *t);

/* psi chosen for prime `index` of the tables (host read, for checking). */
he_status he_ntt_tables_psi(const he_ntt_tables *t, uint32_t index, uint64_t *psi_out);

/* ---- transforms and products (Sec. II-B, Sec. III-B) ------------------------- */

/* Forward negacyclic NTT, in place, of `count` polynomials of `limbs` limbs
 * each, stored back to back (poly[(p * limbs + l) * N + i]); limb l uses prime
 * l of the tables, which must hold at least `limbs` primes equal to
 * moduli_host[0..limbs-1] (checked on the host). Natural-order coefficients
 * become evaluations in bit-reversed order:
 *     out[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q.
 * The psi twist of Sec. II-B is folded into the twiddles. */
he_status he_ntt_fwd(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                     const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream);

/* Inverse negacyclic NTT (Sec. II-B), in place, including the factor N^-1, so that
 * he_ntt_inv(he_ntt_fwd(a)) = a exactly. Same layout and checks. */
he_status he_ntt_inv(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                     const uint64_t *moduli_host, const he_ntt_tables *tw, he_stream_t stream);

/* The naive radix-2 transform of Sec. III-B (one launch per stage, every
 * stage through global memory): the paper's baseline, kept for comparison.
 * Same contract as he_ntt_fwd / he_ntt_inv. */
he_status he_ntt_fwd_naive(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                           const uint64_t *moduli_host, const he_ntt_tables *tw,
                           he_stream_t stream);
he_status he_ntt_inv_naive(uint64_t *poly, uint32_t N, uint32_t limbs, uint32_t count,
                           const uint64_t *moduli_host, const he_ntt_tables *tw,
                           he_stream_t stream);

/* Transform shapes built for degree N: writes up to `cap` triples
 * (log_block, log_thread_words, ctas_per_sm) to shapes_out (host, 3 x cap
 * words), the default first, and the number built to *n_out. log_block:
 * 2^log_block words per CTA, the transform of one limb split over a cluster
 * of N / 2^log_block CTAs; log_thread_words: 2^log_thread_words words per
 * thread, i.e. radix-2^k register rounds (the paper's radix and SLM-stage
 * choices, Sec. III-B); ctas_per_sm: the CTAs per SM the transform kernels
 * are compiled for, i.e. their register budget (0 = the shape's default). */
he_status he_ntt_shapes(uint32_t N, uint32_t *shapes_out, uint32_t cap, uint32_t *n_out);

/* Shape used from now on by he_ntt_fwd (direction 1), he_ntt_inv (2) or
 * both (0) at degree N (process wide; all zero restores the built-in
 * default). persistent != 0 launches a fixed grid of as many clusters as fit
 * on the GPU, each walking over the limbs, instead of one cluster per limb;
 * ctas_per_sm selects a build of the shape for that register budget (0 =
 * default; he_ntt_shapes lists the builds). The autotuner's choices are
 * applied here. Returns HE_EUNSUPPORTED for a shape that is not built. */
he_status he_ntt_set_shape(uint32_t N, uint32_t direction, uint32_t log_block, uint32_t log_thread_words,
                           uint32_t persistent, uint32_t ctas_per_sm);

/* Dyadic product out[l][i] = a[l][i] * b[l][i] mod q_l for `count`
 * polynomials of `limbs` limbs (Sec. II-B, the elementwise product of the
 * convolution theorem). out may equal a or b. */
he_status he_dyadic_mul(uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t N,
                        uint32_t limbs, uint32_t count, const uint64_t *moduli_host,
                        const he_ntt_tables *tw, he_stream_t stream);

/* Negacyclic product c = a * b mod (X^N + 1, q_l), coefficient domain in and
 * out, for `count` polynomials of `limbs` limbs (Sec. II-B: the product is
 * INTT(NTT(a) . NTT(b))), fused into ONE launch: per limb, one cluster runs
 * both forward transforms, the pointwise product and the inverse transform
 * with the data on chip (16 bytes read and 8 written per word, against 72
 * for he_ntt_fwd x 2 + he_dyadic_mul + he_ntt_inv). The transform shape is
 * the forward shape set for N (he_ntt_set_shape). c may equal a or b; any
 * other overlap is HE_EINVAL. Same layout and checks as he_ntt_fwd. */
he_status he_negacyclic_mul(uint64_t *c, const uint64_t *a, const uint64_t *b, uint32_t N,
                            uint32_t limbs, uint32_t count, const uint64_t *moduli_host,
                            const he_ntt_tables *tw, he_stream_t stream);

/* ---- CKKS evaluation (Sec. II-A) ------------------------------------------- */

/* A modulus chain (the RNS representation of Sec. II-B; levels and the
 * special prime of key switching, Sec. II-A): n_data data primes q_0..q_L
 * (L = n_data - 1, n_data <= 32) and one special prime P, all distinct,
 * 2^30 <= q < 2^60, q = 1 mod 2N. Builds the
 * NTT tables of all n_data + 1 primes and the constants of key switching and
 * rescaling. Synchronises. */
he_status he_context_create(uint32_t N, uint32_t n_data, const uint64_t *data_moduli_host,
                            uint64_t special_modulus, he_context **out);
he_status he_context_destroy(he_context *ctx);

/* Words per thread of the context's key-switching and rescale kernels:
 * 2^3 (radix-8 register rounds) or 2^4 (radix-16, the default; 0 restores
 * it). The autotuner times both. */
he_status he_context_set_eval_shape(he_context *ctx, uint32_t log_thread_words);

/* Upload a relinearization key (the evk of Relin, Sec. II-A; a Galois key
 * for he_rotate has the same layout). evk_host is [n_data][2][n_data + 1][N] in the
 * NTT domain: digit j, component k, limbs q_0..q_L then P; it must satisfy
 * evk[j][0] + evk[j][1] s = e_j + [j = i] (P mod q_i) s^2 on limb q_i (and no
 * s^2 term on P), i.e. one RNS digit per data prime and one special prime.
 * The device copy stores each word with its Shoup quotient. Synchronises. */
he_status he_relin_key_upload(const he_context *ctx, const uint64_t *evk_host,
                              he_relin_key **out);
he_status he_relin_key_destroy(he_relin_key *key);

/* Mul (Sec. II-A): out3 = (a0 b0, a0 b1 + a1 b0, a1 b1) mod q_i for the
 * level-l ciphertexts ct_a and ct_b ([2][l+1][N]); out3 is [3][l+1][N]. The
 * middle term takes one reduction (the mad_mod of Sec. III-A-1). */
he_status he_ct_mul(uint64_t *out3, const uint64_t *ct_a, const uint64_t *ct_b,
                    const he_context *ctx, uint32_t level, he_stream_t stream);

/* Relin (Sec. II-A): ct_out2 = (c0, c1) + round(P^-1 c[2] evk) mod q_l, with
 * c[2] split into its RNS digits [c[2]]_{q_j} in [0, q_j) and the division by
 * P rounded half up. ct_in3 is [3][l+1][N], ct_out2 is [2][l+1][N].
 *
 * Scratch (device, 32-byte aligned, contents irrelevant) of key switching,
 * with n = l + 1 limbs: at least (3 n + 2) N words (Relin) or
 * (3 n + 4) N words per pair (MulLinRS); then the mod-up runs as one fused
 * kernel per (ciphertext, target prime). With room for (n + 1) n N more
 * words per ciphertext of a group of up to 64 the mod-up is expanded: each
 * digit-to-target transform runs as its own cluster at the plain
 * transform's size, and the key products as an elementwise pass -- faster,
 * same result. The *_scratch_bytes functions return the expanded size. */
size_t he_relin_scratch_bytes(const he_context *ctx, uint32_t level);
he_status he_relin(uint64_t *ct_out2, const uint64_t *ct_in3, const he_relin_key *key,
                   const he_context *ctx, uint32_t level, void *scratch, size_t scratch_bytes,
                   he_stream_t stream);

/* RS (Sec. II-A): ct_out = round(ct_in / q_l) mod q_0..q_{l-1}, rounded half
 * up; ct_in is [2][l+1][N], ct_out is [2][l][N], level >= 1. */
size_t he_rescale_scratch_bytes(const he_context *ctx, uint32_t level);
he_status he_rescale(uint64_t *ct_out, const uint64_t *ct_in, const he_context *ctx,
                     uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream);

/* MulLinRS (Sec. IV-C): Mul, Relin and RS of `count` ciphertext pairs in one
 * fused sequence of launches. ct_a, ct_b are [count][2][l+1][N]; ct_out is
 * [count][2][l][N]. The two roundings (by P, then by q_l) stay separate, so
 * the result equals he_rescale(he_relin(he_ct_mul(a, b))). */
size_t he_mul_relin_rescale_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count);
/* Scratch bytes for `count` pairs with the mod-up expanded in groups of at
 * most expand_group ciphertexts (0: the fused mod-up's minimum); the plain
 * query above uses groups of 64. Smaller groups trade speed for memory. */
size_t he_mul_relin_rescale_scratch_bytes_ex(const he_context *ctx, uint32_t level, uint32_t count,
                                             uint32_t expand_group);
he_status he_mul_relin_rescale(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b,
                               uint32_t count, const he_relin_key *key, const he_context *ctx,
                               uint32_t level, void *scratch, size_t scratch_bytes,
                               he_stream_t stream);

/* ---- the other routines of Sec. IV-C and the matrix product of Sec. IV-E ---------- */

/* SqrLinRS: the square of each ciphertext (tensor (a0^2, 2 a0 a1, a1^2)),
 * relinearized and rescaled; equals he_mul_relin_rescale(a, a). ct_a is
 * [count][2][l+1][N], ct_out [count][2][l][N]; scratch as MulLinRS. */
he_status he_sqr_relin_rescale(uint64_t *ct_out, const uint64_t *ct_a, uint32_t count,
                               const he_relin_key *key, const he_context *ctx, uint32_t level,
                               void *scratch, size_t scratch_bytes, he_stream_t stream);

/* MulLin (Sec. IV-C routine set): Mul then Relin of `count` pairs, no rescale: ct_out
 * [count][2][l+1][N] equals he_relin(he_ct_mul(a, b)). Scratch: at least
 * (3 n + 2) N words per pair; he_mul_relin_scratch_bytes also makes room
 * for the expanded mod-up (groups of up to 64). */
size_t he_mul_relin_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count);
he_status he_mul_relin(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b, uint32_t count,
                       const he_relin_key *key, const he_context *ctx, uint32_t level, void *scratch,
                       size_t scratch_bytes, he_stream_t stream);

/* Relin then RS (Sec. II-A; the lazy relinearization of the matrix product,
 * Sec. IV-E) of `count` three-component ciphertexts ct3
 * [count][3][l+1][N] (for instance tensors accumulated over a matrix
 * product, relinearized once per output), into [count][2][l][N]; equals
 * he_rescale(he_relin(ct3)). Scratch as MulLinRS. */
he_status he_relin_rescale(uint64_t *ct_out, const uint64_t *ct3, uint32_t count, const he_relin_key *key,
                           const he_context *ctx, uint32_t level, void *scratch, size_t scratch_bytes,
                           he_stream_t stream);

/* Add (Sec. II-A): ct_out = ct_a + ct_b mod q_i, `count` ciphertexts of
 * `components` (2 or 3) components at level l ([count][components][l+1][N]).
 * ct_out may equal ct_a or ct_b. */
he_status he_ct_add(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b, uint32_t count,
                    uint32_t components, const he_context *ctx, uint32_t level, he_stream_t stream);

/* The automorphism X -> X^galois_elt (odd, below 2N; the first step of
 * Rotate, Sec. IV-C) applied to each of
 * `components` components of `count` level-l ciphertexts in the NTT domain
 * ([count][components][l+1][N]); a permutation of every limb's evaluations.
 * Not in place. */
he_status he_ct_automorph(uint64_t *ct_out, const uint64_t *ct_in, uint32_t count, uint32_t components,
                          uint32_t galois_elt, const he_context *ctx, uint32_t level, he_stream_t stream);

/* Rotate (Sec. IV-C routine set): for each of `count` level-l ciphertexts
 * ([count][2][l+1][N] in and out), (sigma(c0), sigma(c1)) with
 * sigma: X -> X^galois_elt, then sigma(c1) key-switched back to s with the
 * Galois key, i.e. he_relin of (sigma(c0), 0, sigma(c1)). galois_elt = 5^k
 * mod 2N rotates the slots by k (slot j at zeta^(5^j)); 2N - 1 conjugates.
 * The Galois key has the relinearization key's layout and is uploaded with
 * he_relin_key_upload: evk[j][0] + evk[j][1] s = e_j + [j = i] (P mod q_i)
 * s(X^galois_elt) on limb q_i (no such term on P). Scratch:
 * he_rotate_scratch_bytes (at least 3 n N + (3 n + 2) N words per
 * ciphertext). */
size_t he_rotate_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count);
he_status he_rotate(uint64_t *ct_out, const uint64_t *ct_in, uint32_t count, uint32_t galois_elt,
                    const he_relin_key *galois_key, const he_context *ctx, uint32_t level, void *scratch,
                    size_t scratch_bytes, he_stream_t stream);

/* Tensor part of the encrypted matrix product C += A B (Sec. IV-E,
 * matMul_mxnxk): for the m x k matrix A and the k x n matrix B of level-l
 * ciphertexts (row-major, each [2][l+1][N]), t_out[i][j] (row-major m x n,
 * each [3][l+1][N]) = sum over l' of the tensor of A[i][l'] and B[l'][j]
 * (Sec. II-A Mul, accumulated before relinearization). he_relin_rescale of
 * t_out followed by he_ct_add into C completes C += A B with one key switch
 * per output (lazy relinearization). m, n, k >= 1. */
he_status he_ct_matmul_tensor(uint64_t *t_out, const uint64_t *a, const uint64_t *b, uint32_t m, uint32_t k,
                              uint32_t n, const he_context *ctx, uint32_t level, he_stream_t stream);

/* Allocation-free MulLinRS: the same result as he_mul_relin_rescale. The
 * paper has no counterpart; this entry point exists for callers that cannot
 * allocate device memory when they need the routine -- code running during
 * stream capture, latency-critical serving
 * paths that must not block on the device allocator, and embedders whose
 * device memory is budgeted by another runtime. It computes exactly what
 * he_mul_relin_rescale computes (same arguments minus the scratch buffer),
 * taking its scratch from a buffer of HE_NOALLOC_SCRATCH_BYTES compiled into
 * the library, held on every GPU that loads the library until the process
 * exits. It never allocates. Requests needing more scratch than that
 * ((3 (level + 1) + 4) * N * 8 bytes per pair, the fused mod-up's minimum)
 * return HE_EINVAL with a message; the expanded mod-up runs when the
 * buffer also holds its group buffer. The first call on each device (and
 * the first after that device's context was destroyed and re-created, e.g. by
 * cudaDeviceReset) resolves the buffer's address (cudaGetSymbolAddress, with
 * that device current); the address is cached per context, so make that first
 * call before any stream capture. All calls share the buffer: calls that may
 * overlap on the GPU race and must be ordered by the caller (e.g. one
 * stream). No scratch word needs to start at zero. */
#define HE_NOALLOC_SCRATCH_BYTES (16u << 20)
he_status he_mul_relin_rescale_noalloc(uint64_t *ct_out, const uint64_t *ct_a, const uint64_t *ct_b,
                                       uint32_t count, const he_relin_key *key, const he_context *ctx,
                                       uint32_t level, he_stream_t stream);

/* ---- mixed-level batches (Sec. III-B batching over instances) ---------------- */

/* One job of a mixed-level MulLinRS batch: `count` ciphertext pairs at
 * `level` (ct_a, ct_b: count x 2 x (level + 1) x N words, NTT domain; ct_out:
 * count x 2 x level x N words), all under one context and key. */
typedef struct he_mrr_job {
    uint64_t *ct_out;
    const uint64_t *ct_a;
    const uint64_t *ct_b;
    uint32_t count;
    uint32_t level;
} he_mrr_job;

/* Device scratch of he_mul_relin_rescale_batch for these jobs (host array):
 * per job count * (level + 3)^2 * N * 8 bytes (the expanded
 * mod-up buffer of all its pairs included). 0 for invalid jobs. */
size_t he_mul_relin_rescale_batch_scratch_bytes(const he_context *ctx, const he_mrr_job *jobs_host,
                                                uint32_t n_jobs);

/* MulLinRS (Sec. IV-C) of every job, each with exactly the result he_mul_relin_rescale
 * gives for it alone, with ONE launch per pipeline stage for all jobs
 * together (digit INTT, mod-up transforms, key multiply-accumulate, the
 * special prime's INTT, and the three mod-down / rescale kernels): the
 * kernels read a table of the jobs (at most 16 per pass; more jobs take
 * further passes) and map each CTA or thread to its job. Jobs may have
 * different levels and counts; jobs with count 0 are skipped. Outputs must
 * not overlap inputs or each other. scratch: device, 32-byte aligned,
 * he_mul_relin_rescale_batch_scratch_bytes. HE_EINVAL for a bad level (< 1
 * or beyond the chain), pointer, key, short scratch, or a batch whose item
 * count exceeds the launch limits. */
he_status he_mul_relin_rescale_batch(const he_mrr_job *jobs_host, uint32_t n_jobs, const he_relin_key *key,
                                     const he_context *ctx, void *scratch, size_t scratch_bytes,
                                     he_stream_t stream);

/* ---- multi-degree batches (Sec. III-B batching over instances) ---------------- */

/* One job of a multi-degree MulLinRS batch: `count` ciphertext pairs at
 * `level` under their own context and relinearization key (ct_a, ct_b:
 * count x 2 x (level + 1) x N words, NTT domain; ct_out: count x 2 x level
 * x N words; N is the context's degree). */
typedef struct he_mrr_multi_job {
    uint64_t *ct_out;
    const uint64_t *ct_a;
    const uint64_t *ct_b;
    uint32_t count;
    uint32_t level;
    const he_context *ctx;
    const he_relin_key *key;
} he_mrr_multi_job;

/* Device scratch of he_mul_relin_rescale_multi for these jobs (host array):
 * per job (level + 3)^2 x N x count x 8 bytes, N its context's degree.
 * 0 for invalid jobs. */
size_t he_mul_relin_rescale_multi_scratch_bytes(const he_mrr_multi_job *jobs_host, uint32_t n_jobs);

/* MulLinRS (Sec. IV-C) of jobs of DIFFERENT degrees, each with exactly the
 * result he_mul_relin_rescale gives for it alone, with ONE launch per
 * pipeline stage for all of them (digit INTT, mod-up transforms, key
 * multiply-accumulate, the special prime's INTT, and the three mod-down /
 * rescale kernels; Sec. II-A Mul, Relin, RS). Each job names its context
 * (degree N in [2^12, 2^15], HE_EUNSUPPORTED otherwise) and a key of that
 * context; levels and counts may differ; count-0 jobs are skipped; at most
 * 16 jobs per pass, more take further passes. The transform stages run
 * clusters of 8 CTAs of 2^12 words, each holding 8 >> c items of a job of
 * degree 2^(12 + c). Outputs must not overlap inputs or each other.
 * scratch: device, 32-byte aligned, he_mul_relin_rescale_multi_scratch_bytes.
 * HE_EINVAL for a bad context, key, level (< 1 or beyond the chain),
 * pointer, short scratch, or a batch beyond the launch limits. */
he_status he_mul_relin_rescale_multi(const he_mrr_multi_job *jobs_host, uint32_t n_jobs, void *scratch,
                                     size_t scratch_bytes, he_stream_t stream);

/* ---- encoding and decoding (Sec. II-A Encode / Decode) ------------------------ */

/* Slot vectors are n = N/2 complex numbers, stored as interleaved FP64
 * (re, im) pairs: slots[(c * n + j) * 2 + {0, 1}] for message c. Slot j is
 * the value of the plaintext polynomial m at the root zeta^(5^j mod 2N),
 * zeta = exp(i pi / N) (Sec. II-A: the canonical embedding restricted to one
 * root of each conjugate pair). The paper encodes and decodes on the host
 * (Sec. III); these calls do it on the device with an FP64 FFT of n points. */
typedef struct he_encoder he_encoder;    /* FFT and CRT tables of a context */

/* Builds the encoding tables (Sec. II-A) for every level of `ctx` (which must outlive the
 * encoder). Synchronises. */
he_status he_encoder_create(const he_context *ctx, he_encoder **out);
he_status he_encoder_destroy(he_encoder *enc);

/* Device scratch of he_encode / he_decode for `count` messages at `level`:
 * encode count * N * 8 bytes; decode count * (level + 3) * N * 8 bytes. */
size_t he_encode_scratch_bytes(const he_encoder *enc, uint32_t count);
size_t he_decode_scratch_bytes(const he_encoder *enc, uint32_t level, uint32_t count);

/* Encode (Sec. II-A): for each of `count` messages, the real polynomial m with
 * m(zeta^(5^j)) = scale * slots_j and m(zeta^(-5^j)) = its conjugate,
 * rounded coefficient by coefficient to the nearest integer (ties to even),
 * reduced modulo q_0..q_level and transformed to the NTT domain:
 * pt_out[(c * (level + 1) + l) * N + i] (the layout of a ciphertext
 * component). The FFT rounds like any FP64 computation: a coefficient whose
 * exact value lies within about 2^-52 * scale * max|slots| * log2(N) of a
 * half-integer may round to either neighbour. scale must be finite and
 * positive and every scaled coefficient below 2^62 in magnitude (larger
 * ones give unspecified residues). slots: device, count * N/2 pairs;
 * scratch: he_encode_scratch_bytes. HE_EINVAL for a bad level, scale,
 * pointer or short scratch. */
he_status he_encode(const he_encoder *enc, uint64_t *pt_out, const double *slots, uint32_t count,
                    double scale, uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream);

/* Decode (Sec. II-A): the inverse NTT of each plaintext pt[c] (count messages of
 * level + 1 limbs, NTT domain, canonical), the CRT lift of every
 * coefficient to the centred integer in [-(Q-1)/2, (Q-1)/2], Q = q_0 ...
 * q_level, its nearest double, the slot values m(zeta^(5^j)) of that real
 * polynomial (FP64 FFT), divided by scale, into slots_out (device,
 * count * N/2 pairs). pt is not modified. A coefficient beyond the double
 * range becomes +-inf. scratch: he_decode_scratch_bytes. */
he_status he_decode(const he_encoder *enc, double *slots_out, const uint64_t *pt, uint32_t count,
                    double scale, uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream);

/* The CRT step of decoding (Sec. II-A, Sec. II-B RNS) alone: out[c * N + i] = the nearest double
 * (round to nearest even) of the centred integer whose residues modulo
 * q_0..q_level are coeffs[(c * (level + 1) + l) * N + i] (coefficient
 * domain, canonical). out and coeffs are device buffers, 8-byte aligned
 * and 32-byte aligned respectively. */
he_status he_crt_compose(const he_encoder *enc, double *out, const uint64_t *coeffs, uint32_t count,
                         uint32_t level, he_stream_t stream);

/* ---- encryption (Sec. II-A Encrypt) ------------------------------------------ */

/* Device scratch of he_encrypt: count * 3 * (level + 1) * N * 8 bytes. */
size_t he_encrypt_scratch_bytes(const he_context *ctx, uint32_t level, uint32_t count);

/* Public-key encryption of `count` plaintexts at `level` (Sec. II-A):
 *   c0 = v pk0 + m + e0,  c1 = v pk1 + e1  (mod q_0 .. q_level),
 * with the products in the NTT domain. pt: count x (level + 1) x N words,
 * NTT domain (he_encode's output); pk: the public key (pk0, pk1) as
 * 2 x n_data x N words in the NTT domain, of which limbs 0..level are used;
 * v, e0, e1: count x N signed 8-bit values each (device), the random
 * ternary mask and the two error polynomials (any |x| < 2^7; the caller
 * draws them, e.g. uniform {-1, 0, 1} and a rounded Gaussian of sigma 3.2);
 * ct_out: count x 2 x (level + 1) x N words. scratch: he_encrypt_scratch_bytes.
 * HE_EINVAL for a bad level, pointer or short scratch. */
he_status he_encrypt(uint64_t *ct_out, const uint64_t *pt, const uint64_t *pk, const int8_t *v,
                     const int8_t *e0, const int8_t *e1, uint32_t count, const he_context *ctx,
                     uint32_t level, void *scratch, size_t scratch_bytes, he_stream_t stream);

/* The encryption randomness drawn on the device (Sec. II-A Encrypt: the
 * ternary mask v and the errors e0, e1 of each message), count x N signed
 * 8-bit values each (device). Generator: SplitMix64 in counter form (Steele,
 * Lea and Flood 2014), output k of stream `seed` = mix(seed + (k + 1) *
 * 0x9E3779B97F4A7C15) with mix(z): z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9;
 * z = (z ^ z >> 27) * 0x94D049BB133111EB; z ^ z >> 31. Draw w (0: v, 1: e0,
 * 2: e1) of message c at coefficient i uses output (3 c + w) N + i, r:
 * v = (r mod 3) - 1; e = popcount(r & (2^20 - 1)) - popcount((r >> 20) &
 * (2^20 - 1)), the centred binomial distribution of parameter 20 (variance
 * 10, |e| <= 20; the paper asks only for Gaussian-distributed errors).
 * Integer-only, so any implementation of this definition reproduces the
 * draws bit for bit. HE_EINVAL for a bad degree or NULL pointer. */
he_status he_sample_encryption_draws(int8_t *v, int8_t *e0, int8_t *e1, uint32_t count, uint32_t N,
                                     uint64_t seed, he_stream_t stream);

/* he_encrypt with its randomness drawn on the device from `seed`: the same
 * ciphertexts as he_encrypt given he_sample_encryption_draws(seed)'s draws
 * (the draws are generated inside the residue kernel, never stored). Same
 * arguments and checks as he_encrypt otherwise. */
he_status he_encrypt_seeded(uint64_t *ct_out, const uint64_t *pt, const uint64_t *pk, uint64_t seed,
                            uint32_t count, const he_context *ctx, uint32_t level, void *scratch,
                            size_t scratch_bytes, he_stream_t stream);

/* ---- batched plans (Sec. III-B parallelism over limbs and instances) -------- */

/* One polynomial of a batched NTT: `limbs` limbs of degree N at `data`
 * (device), limb l using prime (first_prime + l) of `tables`. */
typedef struct he_poly_desc {
    uint64_t *data;
    const he_ntt_tables *tables;
    uint32_t N;
    uint32_t limbs;
    uint32_t first_prime;
    uint32_t reserved;
} he_poly_desc;

/* Kernel shape of a plan for one N: 2^log_block words per CTA (the rest of
 * the transform is split over a cluster of N / 2^log_block CTAs exchanging
 * through distributed shared memory) and 2^log_thread_words words per
 * thread (radix-2^log_thread_words register rounds; 0 = 16 words);
 * persistent != 0 launches a fixed grid of co-resident clusters walking the
 * degree's limbs instead of one cluster per limb (the default, measured
 * faster). */
typedef struct he_ntt_shape {
    uint32_t N;
    uint32_t log_block;
    uint32_t log_thread_words;
    uint32_t persistent;
    uint32_t ctas_per_sm;       /* 0: the shape's default register budget */
} he_ntt_shape;

/* A plan (Sec. III-B parallelism over limbs and instances) that transforms
 * all `count` polynomials (any mix of N and limb
 * counts) with kernels driven by a device-resident work list. Without shape
 * overrides (n_shapes = 0) and with every N in [2^12, 2^15], the whole plan
 * is ONE launch per direction: one cluster of 8 CTAs per unit of work (8
 * limbs of 2^12, 4 of 2^13, 2 of 2^14 or 1 of 2^15), split into
 * sub-clusters per degree. With overrides (e.g. the autotuner's choices per
 * N), each degree gets its own launch in the given shape. Allocates the
 * work list and synchronises; execution allocates nothing. */
he_status he_ntt_plan_create(const he_poly_desc *descs_host, uint32_t count,
                             const he_ntt_shape *shapes_host, uint32_t n_shapes,
                             he_plan **out);
he_status he_ntt_plan_fwd(const he_plan *plan, he_stream_t stream);
he_status he_ntt_plan_inv(const he_plan *plan, he_stream_t stream);
he_status he_plan_destroy(he_plan *plan);

/* Number of kernel launches one execution of the plan enqueues. */
uint32_t he_plan_launches(const he_plan *plan);

/* ---- host-resident batches (Sec. III asynchronous pipeline, multiple queues) -- */

#define HE_NTT_OP_FORWARD 1u
#define HE_NTT_OP_INVERSE 2u

/* Transforms (Sec. III asynchronous pipeline) `count` polynomials of `limbs` limbs that live in HOST memory
 * (same layout and checks as he_ntt_fwd): in_host is copied to the device,
 * transformed and copied back to out_host. ops = HE_NTT_OP_FORWARD,
 * HE_NTT_OP_INVERSE or both (forward, then inverse). The batch is cut into
 * chunks of whole polynomials that flow through up to four internal streams,
 * so that the host-to-device copy of one chunk, the kernels of another and
 * the device-to-host copy of a third run at the same time (the paper's
 * asynchronous pipeline: transfers and kernels queued without host
 * synchronisation, over several queues).
 *   work / work_bytes: device scratch owned by the caller, 32-byte aligned,
 *     room for at least one polynomial (limbs * N * 8 bytes); more room
 *     (e.g. 4 x 32 polynomials) gives larger chunks and full overlap.
 *   in_host, out_host: equal (in place) or disjoint, count * limbs * N
 *     words each. Page-locked memory (cudaHostAlloc / cudaHostRegister) is
 *     needed for the copies to overlap and for use under stream capture;
 *     pageable memory works but its copies do not overlap.
 * Asynchronous with respect to the host: the work is ordered after
 * everything already queued on `stream`, and `stream` waits for all of it,
 * so host buffers must stay valid until `stream` has reached this point.
 * Calls from several threads are serialised on the internal streams.
 * Returns HE_EINVAL for a bad ops value, NULL or partly overlapping host
 * buffers, or scratch smaller than one polynomial. Allocates nothing but,
 * on the first call on a device, its internal streams and events. */
he_status he_ntt_host(const uint64_t *in_host, uint64_t *out_host, uint32_t N, uint32_t limbs,
                      uint32_t count, const uint64_t *moduli_host, const he_ntt_tables *tw, uint32_t ops,
                      uint64_t *work, size_t work_bytes, he_stream_t stream);

/* ---- measurement -------------------------------------------------------------- */

/* Integer-throughput probe: blocks x threads threads each run 16 * iters
 * Harvey butterflies (Algorithm 1, 60-bit prime) entirely in registers and
 * write one word to sink[blocks * threads] (device). Timing the launch gives
 * the butterfly rate the integer pipes sustain with no memory traffic, the
 * compute roof against which the transforms are reported. */
he_status he_butterfly_probe(uint64_t *sink, uint32_t blocks, uint32_t threads, uint32_t iters,
                             he_stream_t stream);

/* FP64 throughput probe: blocks x threads threads each run 8 independent
 * chains of `iters` fused multiply-adds in registers (16 FLOP per step) and
 * write one double to sink[blocks * threads] (device). Timing the launch
 * gives the FP64 rate that bounds the slot FFT of he_encode / he_decode. */
he_status he_fp64_probe(double *sink, uint32_t blocks, uint32_t threads, uint32_t iters, he_stream_t stream);

/* The transform butterflies applied elementwise to device arrays of n
 * entries, for checking their contract (Algorithm 1) on the device. Forward
 * (inverse = 0): for x, y in [0, 8p + 2^32), w < p and w_shoup =
 * floor(w 2^64 / p), x' = x + w y and y' = x - w y (mod p), both again in
 * [0, 8p + 2^32). Inverse (inverse = 1): for x, y in [0, 4p),
 * x' = x + y and y' = (x - y) w (mod p), both in [0, 4p). 2^30 <= p < 2^60,
 * p need not be prime. x and y are updated in place. */
he_status he_butterfly_apply(uint64_t *x, uint64_t *y, const uint64_t *w, const uint64_t *w_shoup,
                             uint32_t n, uint64_t p, int32_t inverse, he_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HE_H */
