// multi.cu -- MulLinRS over jobs of different degrees (2^12 .. 2^15), each
// with its own context and key, with ONE launch per pipeline stage for all
// of them (Sec. III-B: parallelism over instances, here across degrees too).
//
// Every stage kernel runs clusters of 8 CTAs of 2^12 words each. A cluster
// takes one unit of work: for a job of degree 2^(12 + c), a unit holds up to
// 8 >> c items of the stage, each transformed by a sub-cluster of 2^c CTAs
// (cluster ranks rbase .. rbase + 2^c - 1), the layout of the mixed-degree
// transform (k_ntt_mixed). Units never mix jobs, so all CTAs of a cluster
// run the same transform shape and pass the same cluster barriers; a
// sub-cluster without an item of its own in a job's last unit recomputes the
// unit's first item with every store switched off. The per-item work is the
// stage body shared with the per-degree kernels (kernels.cuh), so results
// are those of he_mul_relin_rescale bit for bit.
#include <mutex>

#include "kernels.cuh"

namespace he {

constexpr u32 kMultiSmem = 4096 * 8;   // one 2^12-word block per CTA

__device__ __forceinline__ int multi_slot(MultiStage S)
{
    switch (S) {
    case MS_DIGITS: return JS_DIGITS;
    case MS_EXPAND: return JS_EXPAND;
    case MS_PLIFT: return JS_PLIFT;
    case MS_LAST: return JS_LAST;
    default: return JS_REST;
    }
}

// Items of stage S for the job bound into a.
template <MultiStage S>
__device__ __forceinline__ u32 multi_items(const EvalArgs &a)
{
    if constexpr (S == MS_DIGITS) return a.count * a.n;
    if constexpr (S == MS_EXPAND) return a.count * a.n * a.n;   // off-diagonal (target, digit) pairs
    if constexpr (S == MS_PLIFT || S == MS_LAST) return 2 * a.count;
    return 2 * a.count * (a.n - 1);
}

// Not inlined: each degree's body gets its own register allocation, where
// one function holding all four shapes spilled heavily at 64 registers.
template <MultiStage S, class Sh>
__device__ __noinline__ void multi_item(const EvalArgs &a, u32 item, u32 m, u32 rbase, bool valid)
{
    if constexpr (S == MS_DIGITS) {
        ks_digits_body<Sh>(a, item, m, rbase, valid);
    } else if constexpr (S == MS_EXPAND) {
        // per ciphertext g: n targets q_t with the n - 1 digits j != t, then
        // the special prime with all n digits
        const u32 n = a.n, nn = n * n;
        const u32 g = item / nn, r = item % nn;
        u32 t, j;
        if (r < n * (n - 1)) {
            t = r / (n - 1);
            const u32 jj = r % (n - 1);
            j = jj + (jj >= t ? 1u : 0u);
        } else {
            t = n;
            j = r - n * (n - 1);
        }
        ks_expand_body<Sh>(a, g, t, j, m, rbase, valid);
    } else if constexpr (S == MS_PLIFT) {
        plift_intt_body<Sh>(a, item, m, rbase, valid);
    } else if constexpr (S == MS_LAST) {
        mrr_last_body<Sh>(a, item, m, rbase, valid);
    } else if constexpr (S == MS_REST_Z) {
        mrr_rest_z_body<Sh>(a, item, m, rbase, valid);
    } else {
        mrr_rest_out_body<Sh>(a, item, m, rbase, valid);
    }
}

// The forward-and-inverse stage keeps more state: the evaluation kernels'
// 128-register budget (two CTAs per SM), the others the transform's 64.
template <MultiStage S>
__global__ void __launch_bounds__(256, S == MS_LAST ? 2 : 4) k_mrr_multi(EvalArgs a0, JobTable t)
{
    EvalArgs a = a0;
    const u32 rank = cluster_ctarank();
    const u32 unit = bind_job(a, t, multi_slot(S), blockIdx.x >> 3);
    const u32 c = (31u - __clz(a.ctx.N)) - 12u;      // 0 .. 3, checked on the host
    const u32 per = 8u >> c;
    const u32 sub = rank >> c;
    const u32 m = rank & ((1u << c) - 1u);
    u32 item = unit * per + sub;
    const bool valid = item < multi_items<S>(a);
    if (!valid) item = unit * per;                   // the unit's first item always exists
    switch (c) {
    case 0: multi_item<S, NttShape<12, 0, 4>>(a, item, m, sub << c, valid); break;
    case 1: multi_item<S, NttShape<12, 1, 4>>(a, item, m, sub << c, valid); break;
    case 2: multi_item<S, NttShape<12, 2, 4>>(a, item, m, sub << c, valid); break;
    default: multi_item<S, NttShape<12, 3, 4>>(a, item, m, sub << c, valid); break;
    }
}

template <MultiStage S>
static cudaError_t launch_stage(const EvalArgs &a, const JobTable &t, u32 units, cudaStream_t s)
{
    static std::once_flag f;
    static cudaError_t e = cudaSuccess;
    std::call_once(f, [] {
        e = cudaFuncSetAttribute(k_mrr_multi<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiSmem);
    });
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(units * 8, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = kMultiSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 8;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mrr_multi<S>, a, t);
}

cudaError_t launch_mrr_multi(MultiStage stage, const EvalArgs &a, const JobTable &t, u32 units, cudaStream_t s)
{
    if (!units) return cudaSuccess;
    switch (stage) {
    case MS_DIGITS: return launch_stage<MS_DIGITS>(a, t, units, s);
    case MS_EXPAND: return launch_stage<MS_EXPAND>(a, t, units, s);
    case MS_PLIFT: return launch_stage<MS_PLIFT>(a, t, units, s);
    case MS_LAST: return launch_stage<MS_LAST>(a, t, units, s);
    case MS_REST_Z: return launch_stage<MS_REST_Z>(a, t, units, s);
    case MS_REST_OUT: return launch_stage<MS_REST_OUT>(a, t, units, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace he
