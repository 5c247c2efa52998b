// launch.h -- argument blocks of the kernels and the per-degree launcher
// table (host and device visible). Internal to the library.
#pragma once
#include <cuda.h>   // CUtensorMap (the type only; nothing links the driver library)
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "modarith.cuh"

namespace he {

// One limb of a batched transform (plans): its data, twiddles and constants.
struct LimbJob {
    u64 *data;
    const ulonglong2 *tw_fwd;
    const ulonglong2 *tw_inv;
    const PrimeConst *pc;
};

// A uniform batch (items = count * limbs limbs of one degree, limb l of each
// polynomial using prime first_prime + l of one table set), or a job list.
// tma_store: the forward transform writes its output with bulk tensor
// stores through tmap, the batch viewed as rows of 16 words (128 bytes),
// boxes of 32 rows, 128-byte swizzle (uniform batches, 16 words a thread).
struct NttLaunch {
    u64 *base;
    u32 limbs;
    u32 first_prime;
    u32 items;
    u32 prefetch;               // > 0: each cluster asks L2 for the limb this many items ahead
    const ulonglong2 *tw_fwd;   // [prime][N]
    const ulonglong2 *tw_inv;
    const PrimeConst *pc;       // [prime]
    const LimbJob *jobs;        // non-null: per-item jobs instead of base/limbs
    u32 tma_store;
    CUtensorMap tmap;
};

// Fused negacyclic product c = a b mod (X^N + 1, q) of items = count * limbs
// limbs (limb l of polynomial p at (p limbs + l) N, prime first_prime + l):
// forward transforms of a and b, pointwise product and inverse transform in
// one launch, the data staying on chip in between.
struct NegaLaunch {
    u64 *c;
    const u64 *a, *b;
    u32 limbs;
    u32 items;
    const ulonglong2 *tw_fwd;   // [prime][N]
    const ulonglong2 *tw_inv;
    const PrimeConst *pc;       // [prime]
};

// A unit of the mixed-degree transform: up to 8 >> (log_n - 12)
// limbs of degree 2^log_n, jobs[first_job .. first_job + n_jobs).
struct MixedUnit {
    u32 log_n;
    u32 first_job;
    u32 n_jobs;
    u32 pad;
};

// Mixed-degree transform of N in [2^12, 2^15]: one launch of `clusters`
// clusters of 8 CTAs walking the unit list (mixed.cu; plans launch one
// cluster per unit).
cudaError_t launch_ntt_mixed(const MixedUnit *units, u32 n_units, const LimbJob *jobs, bool inverse, u32 clusters,
                             cudaStream_t s);

// Device view of a modulus chain (q_0..q_{n_data-1}, then P at n_data).
struct DevCtx {
    const ulonglong2 *tw_fwd;   // [n_data + 1][N]
    const ulonglong2 *tw_inv;
    const PrimeConst *pc;       // [n_data + 1]
    // cst[3 i + {0,1,2}] = P^-1 mod q_i, its Shoup quotient, P mod q_i;
    // cst[3 n_data + 3 (l n_data + i) + {0,1,2}] = q_l^-1 mod q_i, Shoup,
    // q_l mod q_i (rescale from level l, i < l);
    // cst[3 n_data + 3 n_data^2 + i] = Shoup quotient of P mod q_i.
    const u64 *cst;
    u32 N;
    u32 n_data;
};

__host__ __device__ inline u32 p_shoup_index(const DevCtx &c, u32 i) { return 3 * c.n_data * (1 + c.n_data) + i; }

struct EvalArgs {
    const u64 *ct_a, *ct_b;     // [count][2][n][N] (fused Mul) or null
    const u64 *ct3;             // [count][3][n][N] or null
    const u64 *ct2;             // [count][2][n][N] rescale input
    u64 *out;
    u64 *c2;                    // scratch [count][n][N]
    u64 *accq;                  // scratch [count][2][n][N]
    u64 *plift;                 // scratch [count][2][N]
    u64 *lift2;                 // scratch [count][2][N]
    const ulonglong2 *evk;      // [n_data][2][n_data + 1][N] (value, Shoup)
    u64 *mx;                    // expanded mod-up scratch [group][n + 1][n][N]
    u32 n;                      // limbs at the current level
    u32 count;
    u32 c_first;                // first ciphertext of the expanded mod-up group
    u32 pad;
    DevCtx ctx;
};

// Mixed-level batches (one context): each launch of the MulLinRS pipeline
// covers every job; job i's items in stage S start at job[i].begin[S].
// Multi-degree batches (a context and key per job, degrees 2^12 .. 2^15):
// the transform stages count units (clusters of 8 CTAs, each running 8 >> c
// items of degree 2^(12 + c) side by side) instead of items, and the special
// prime's inverse transforms are a stage of their own (JS_PLIFT).
enum JobStage { JS_DIGITS = 0, JS_EXPAND, JS_MAC, JS_LAST, JS_REST, JS_PLIFT, JS_COUNT };
constexpr u32 kMaxJobs = 16;
struct EvalJob {
    const u64 *ct_a, *ct_b;     // [count][2][n][N]
    u64 *out;                   // [count][2][n - 1][N]
    u64 *c2, *accq, *plift, *lift2, *mx;   // the job's scratch regions
    const ulonglong2 *evk;      // the job's key
    DevCtx ctx;                 // the job's context
    u32 n, count;
    u32 begin[JS_COUNT];
};
struct JobTable {               // passed by value (kernel parameter space)
    EvalJob job[kMaxJobs];
    u32 n_jobs;
};
struct NoJobs {};
template <bool JOBS>
using JobsArg = typename std::conditional<JOBS, JobTable, NoJobs>::type;

// Stages of the multi-degree MulLinRS pipeline (multi.cu), one launch each
// over `units` clusters; the key multiply-accumulate between the expansion
// and the special-prime transforms is k_ks_mac over the same job table.
enum MultiStage { MS_DIGITS = 0, MS_EXPAND, MS_PLIFT, MS_LAST, MS_REST_Z, MS_REST_OUT, MS_COUNT };
cudaError_t launch_mrr_multi(MultiStage stage, const EvalArgs &a, const JobTable &t, u32 units, cudaStream_t s);

enum EvalKernel {
    EK_KS_DIGITS = 0,
    EK_KS_MODUP,
    EK_KS_EXPAND,
    EK_KS_MODDOWN,
    EK_RS_LIFT,
    EK_RS,
    EK_MRR_LAST,
    EK_MRR_REST_Z,
    EK_MRR_REST_OUT,
    EK_COUNT
};

// Launchers of one polynomial degree N = 2^log_n. A transform shape is
// (log_b, log_e): 2^log_b words per CTA (a cluster of N / 2^log_b CTAs per
// limb) and 2^log_e words per thread (radix-2^log_e register rounds); 0, 0
// picks the degree's default shape.
struct DegreeOps {
    int log_n;
    int default_log_b;
    int default_log_e;
    // Plain transform of a uniform batch or a job list, one cluster per limb.
    cudaError_t (*ntt)(const NttLaunch &a, int log_b, int log_e, bool inverse, cudaStream_t s);
    // Persistent transform over a job list with `grid_clusters` clusters.
    cudaError_t (*ntt_persistent)(const NttLaunch &a, int log_b, int log_e, bool inverse, u32 grid_clusters,
                                  cudaStream_t s);
    // Largest number of co-resident clusters of the persistent kernel.
    int (*max_clusters)(int log_b, int log_e, bool inverse);
    // Evaluation kernels over `items` clusters (the default words per CTA;
    // log_e = 3 or 4 words per thread, 0 = 4); with a job table (MulLinRS
    // kernels only) the items run over every job of a mixed-level batch.
    cudaError_t (*eval)(EvalKernel k, const EvalArgs &a, u32 items, int log_e, const JobTable *jobs,
                        cudaStream_t s);
    // Is the shape built for this degree?
    bool (*has_shape)(int log_b, int log_e);
    // Fused negacyclic product in the given transform shape (0, 0 = default).
    cudaError_t (*negacyclic)(const NegaLaunch &a, int log_b, int log_e, cudaStream_t s);
    // Shapes built for this degree: n pairs (log_b, log_e), default first.
    int n_shapes;
    const int (*shapes)[2];
};

const DegreeOps *degree_ops(int log_n);

// Encoding and decoding (encode.cu): the slot FFT of n = N/2 points in two
// passes (n = n1 n2, n1 = 2^log_n1), fused with the slot permutation and
// scaling at one end and the twist by zeta^k at the other.
struct FftArgs {
    const double2 *z_in;     // encode: slots [count][n]
    double2 *z_out;          // decode: slots [count][n]
    const double *m_in;      // decode: centred coefficients [count][N]
    u64 *pt_out;             // encode: coefficient residues [count][limbs][N]
    double2 *u;              // scratch between the passes [count][n]
    const double2 *omega;    // exp(-2 pi i j / n), j < n
    const double2 *zeta;     // exp(i pi k / N), k < n
    const u32 *slot_of;      // slot j of FFT index t_j = (5^j mod 2N - 1) / 4
    const u64 *primes;       // encode: (q_i, floor(2^64 / q_i)), i < limbs
    double scale;            // encode: Delta; decode: 1 / Delta
    double inv_n;            // 1 / n
    u32 log_n, log_n1, limbs, count;
};
cudaError_t launch_encode_fft(const FftArgs &a, cudaStream_t s);
cudaError_t launch_decode_fft(const FftArgs &a, cudaStream_t s);
// Words of the CRT kernel's multi-word integers for `need` words (0: too many).
u32 crt_words(u32 need);
cudaError_t launch_crt_compose(double *out, const u64 *coef, const u64 *tab, u32 nw, u32 log_N, u32 limbs, u64 total,
                               u32 blocks, cudaStream_t s);

}  // namespace he
