// inst.cuh -- per-degree instantiation of the kernels and their launchers.
// Each inst_n<log N>.cu includes this file and lists the shapes of its
// degree, so that the degrees compile as separate translation units, in
// parallel.
#pragma once
#include <mutex>

#include "kernels.cuh"

namespace he {

template <class K, class... Args>
static cudaError_t launch_k(K kernel, u32 grid, u32 block, u32 smem, u32 cluster, cudaStream_t s,
                            Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.numAttrs = 0;
    if (cluster > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Raise the dynamic shared-memory limit of a kernel once per process, and
// allow its launch in clusters of more than 8 CTAs (the non-portable size,
// up to 16 on this GPU) where the shape needs it.
template <class K>
static cudaError_t smem_attr(K kernel, u32 bytes, std::once_flag &flag, cudaError_t &err, u32 cluster = 0)
{
    std::call_once(flag, [&] {
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (err == cudaSuccess && cluster > 8)
            err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
    return err;
}

// OCC: CTAs per SM of the plain and persistent transform kernels (their
// register budget; 0 = the shape's default); the other kernels of a shape do
// not depend on it.
template <int LOG_B, int LOG_C, int LOG_E = 4, int OCC = 0>
struct ShapeOps {
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;

    template <bool INV>
    static cudaError_t ntt(const NttLaunch &a, cudaStream_t s)
    {
        static std::once_flag f;
        static cudaError_t e = cudaSuccess;
        if (cudaError_t r = smem_attr(k_ntt<LOG_B, LOG_C, LOG_E, INV, OCC>, Sh::SMEM_BYTES, f, e, Sh::C)) return r;
        return launch_k(k_ntt<LOG_B, LOG_C, LOG_E, INV, OCC>, a.items * Sh::C, Sh::T, Sh::SMEM_BYTES, Sh::C, s, a);
    }

    template <bool INV>
    static cudaError_t persistent(const NttLaunch &a, u32 clusters, cudaStream_t s)
    {
        static std::once_flag f;
        static cudaError_t e = cudaSuccess;
        if (cudaError_t r = smem_attr(k_ntt_persistent<LOG_B, LOG_C, LOG_E, INV, OCC>, Sh::SMEM_BYTES, f, e, Sh::C)) return r;
        return launch_k(k_ntt_persistent<LOG_B, LOG_C, LOG_E, INV, OCC>, clusters * Sh::C, Sh::T, Sh::SMEM_BYTES, Sh::C,
                        s, a);
    }

    static cudaError_t negacyclic(const NegaLaunch &a, cudaStream_t s)
    {
        static std::once_flag f;
        static cudaError_t e = cudaSuccess;
        if (cudaError_t r = smem_attr(k_negacyclic<LOG_B, LOG_C, LOG_E>, 2 * Sh::SMEM_BYTES, f, e, Sh::C)) return r;
        return launch_k(k_negacyclic<LOG_B, LOG_C, LOG_E>, a.items * Sh::C, Sh::T, 2 * Sh::SMEM_BYTES, Sh::C, s, a);
    }

    // Co-resident clusters of the transform (the persistent kernel has the
    // plain kernel's resources), queried once per process.
    template <bool INV>
    static int max_clusters()
    {
        static std::once_flag once;
        static int n = 0;
        std::call_once(once, [] { n = query_max_clusters<INV>(); });
        return n;
    }

    template <bool INV>
    static int query_max_clusters()
    {
        static std::once_flag f;
        static cudaError_t e = cudaSuccess;
        if (smem_attr(k_ntt_persistent<LOG_B, LOG_C, LOG_E, INV, OCC>, Sh::SMEM_BYTES, f, e, Sh::C) != cudaSuccess) return 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(Sh::C * 1024, 1, 1);
        cfg.blockDim = dim3(Sh::T, 1, 1);
        cfg.dynamicSmemBytes = Sh::SMEM_BYTES;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = Sh::C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_ntt_persistent<LOG_B, LOG_C, LOG_E, INV, OCC>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }

    static cudaError_t eval(EvalKernel k, const EvalArgs &a, u32 items, const JobTable *jobs, cudaStream_t s)
    {
        const u32 grid = items * Sh::C;
        const u32 sm1 = Sh::SMEM_BYTES;
        const u32 sm3 = Sh::SMEM_BYTES * 3;    // modup: transform + two accumulators
        switch (k) {
#define HE_EVAL_CASE(ID, KERNEL, SMEM)                                                   \
    case ID: {                                                                           \
        if (jobs) return cudaErrorInvalidValue;                                          \
        static std::once_flag f;                                                         \
        static cudaError_t e = cudaSuccess;                                              \
        if (cudaError_t r = smem_attr(KERNEL<LOG_B, LOG_C, LOG_E>, SMEM, f, e)) return r; \
        return launch_k(KERNEL<LOG_B, LOG_C, LOG_E>, grid, Sh::T, SMEM, Sh::C, s, a);     \
    }
#define HE_EVAL_CASE_J(ID, KERNEL, SMEM)                                                                    \
    case ID: {                                                                                              \
        if (jobs) {                                                                                         \
            static std::once_flag f;                                                                        \
            static cudaError_t e = cudaSuccess;                                                             \
            if (cudaError_t r = smem_attr(KERNEL<LOG_B, LOG_C, LOG_E, true>, SMEM, f, e)) return r;         \
            return launch_k(KERNEL<LOG_B, LOG_C, LOG_E, true>, grid, Sh::T, SMEM, Sh::C, s, a, *jobs);      \
        }                                                                                                   \
        static std::once_flag f;                                                                            \
        static cudaError_t e = cudaSuccess;                                                                 \
        if (cudaError_t r = smem_attr(KERNEL<LOG_B, LOG_C, LOG_E, false>, SMEM, f, e)) return r;            \
        return launch_k(KERNEL<LOG_B, LOG_C, LOG_E, false>, grid, Sh::T, SMEM, Sh::C, s, a, NoJobs{});      \
    }
            HE_EVAL_CASE_J(EK_KS_DIGITS, k_ks_digits, sm1)
            HE_EVAL_CASE(EK_KS_MODUP, k_ks_modup, sm3)
            HE_EVAL_CASE_J(EK_KS_EXPAND, k_ks_expand, sm1)
            HE_EVAL_CASE(EK_KS_MODDOWN, k_ks_moddown, sm1)
            HE_EVAL_CASE(EK_RS_LIFT, k_rs_lift, sm1)
            HE_EVAL_CASE(EK_RS, k_rs, sm1)
            HE_EVAL_CASE_J(EK_MRR_LAST, k_mrr_last, sm1)
            HE_EVAL_CASE_J(EK_MRR_REST_Z, k_mrr_rest_z, sm1)
            HE_EVAL_CASE_J(EK_MRR_REST_OUT, k_mrr_rest_out, sm1)
#undef HE_EVAL_CASE_J
#undef HE_EVAL_CASE
        default:
            return cudaErrorInvalidValue;
        }
    }
};

}  // namespace he

// Shapes built per degree: 2^LB words per CTA (at most 8 CTAs per cluster)
// and 2^LE words per thread. The first listed is the default (and the one
// the evaluation kernels use). Internally a shape's thread-words code is
// LE | OCC << 4, OCC the CTAs per SM its transform kernels are compiled for
// (0: the shape's default budget).
#define HE_SHAPE_FN(LOG_N_, LB, LE)                                                                \
    if (log_b == LB && log_e == LE) return fn(::he::ShapeOps<LB, LOG_N_ - LB, LE>{});
#define HE_SHAPE_FN_OCC(LOG_N_, LB, LE, OCC)                                                       \
    if (log_b == LB && log_e == ((LE) | ((OCC) << 4))) return fn(::he::ShapeOps<LB, LOG_N_ - LB, LE, OCC>{});

namespace he {

template <int LOG_N>
struct DegreeImpl;

#define HE_DEGREE(LOG_N_, DEF_B, DEF_E, LIST, ...)                                                 \
    template <>                                                                                    \
    struct DegreeImpl<LOG_N_> {                                                                    \
        static constexpr int def_b = DEF_B;                                                        \
        static constexpr int def_e = DEF_E;                                                        \
        static constexpr int shapes[][2] = LIST;                                                   \
        template <class F>                                                                         \
        static auto with_shape(int log_b, int log_e, F fn)                                         \
            -> decltype(fn(ShapeOps<DEF_B, LOG_N_ - DEF_B, DEF_E>{}))                              \
        {                                                                                          \
            if (log_b == 0) log_b = DEF_B;                                                         \
            if ((log_e & 15) == 0) log_e |= DEF_E;                                                 \
            __VA_ARGS__                                                                            \
            return decltype(fn(ShapeOps<DEF_B, LOG_N_ - DEF_B, DEF_E>{}))();                       \
        }                                                                                          \
    };

}  // namespace he

#define HE_DEFINE_DEGREE_OPS(LOG_N_)                                                               \
    namespace he {                                                                                 \
    static cudaError_t ntt_##LOG_N_(const NttLaunch &a, int log_b, int log_e, bool inv, cudaStream_t s) \
    {                                                                                              \
        using D = DegreeImpl<LOG_N_>;                                                              \
        bool found = false;                                                                        \
        cudaError_t r = D::with_shape(log_b, log_e, [&](auto ops) {                                \
            found = true;                                                                          \
            return inv ? decltype(ops)::template ntt<true>(a, s) : decltype(ops)::template ntt<false>(a, s); \
        });                                                                                        \
        return found ? r : cudaErrorInvalidValue;                                                  \
    }                                                                                              \
    static cudaError_t ntt_p_##LOG_N_(const NttLaunch &a, int log_b, int log_e, bool inv, u32 cl,   \
                                      cudaStream_t s)                                              \
    {                                                                                              \
        using D = DegreeImpl<LOG_N_>;                                                              \
        bool found = false;                                                                        \
        cudaError_t r = D::with_shape(log_b, log_e, [&](auto ops) {                                \
            found = true;                                                                          \
            return inv ? decltype(ops)::template persistent<true>(a, cl, s)                       \
                       : decltype(ops)::template persistent<false>(a, cl, s);                     \
        });                                                                                        \
        return found ? r : cudaErrorInvalidValue;                                                  \
    }                                                                                              \
    static int maxcl_##LOG_N_(int log_b, int log_e, bool inv)                                      \
    {                                                                                              \
        using D = DegreeImpl<LOG_N_>;                                                              \
        return D::with_shape(log_b, log_e, [&](auto ops) {                                         \
            return inv ? decltype(ops)::template max_clusters<true>()                              \
                       : decltype(ops)::template max_clusters<false>();                           \
        });                                                                                        \
    }                                                                                              \
    static cudaError_t eval_##LOG_N_(EvalKernel k, const EvalArgs &a, u32 items, int log_e,        \
                                     const JobTable *jobs, cudaStream_t s)                         \
    {                                                                                              \
        using D = DegreeImpl<LOG_N_>;                                                              \
        if (log_e == 3) return ShapeOps<D::def_b, LOG_N_ - D::def_b, 3>::eval(k, a, items, jobs, s); \
        return ShapeOps<D::def_b, LOG_N_ - D::def_b, 4>::eval(k, a, items, jobs, s);               \
    }                                                                                              \
    static cudaError_t nega_##LOG_N_(const NegaLaunch &a, int log_b, int log_e, cudaStream_t s)     \
    {                                                                                              \
        using D = DegreeImpl<LOG_N_>;                                                              \
        bool found = false;                                                                        \
        cudaError_t r = D::with_shape(log_b, log_e, [&](auto ops) {                                \
            found = true;                                                                          \
            return decltype(ops)::negacyclic(a, s);                                                \
        });                                                                                        \
        return found ? r : cudaErrorInvalidValue;                                                  \
    }                                                                                              \
    static bool has_##LOG_N_(int log_b, int log_e)                                                 \
    {                                                                                              \
        return DegreeImpl<LOG_N_>::with_shape(log_b, log_e, [&](auto) { return true; });           \
    }                                                                                              \
    extern const DegreeOps degree_ops_##LOG_N_ = {                                                 \
        LOG_N_, DegreeImpl<LOG_N_>::def_b, DegreeImpl<LOG_N_>::def_e, ntt_##LOG_N_, ntt_p_##LOG_N_,  \
        maxcl_##LOG_N_, eval_##LOG_N_, has_##LOG_N_, nega_##LOG_N_,                                \
        (int)(sizeof(DegreeImpl<LOG_N_>::shapes) / sizeof(DegreeImpl<LOG_N_>::shapes[0])),         \
        DegreeImpl<LOG_N_>::shapes};                                                               \
    }
