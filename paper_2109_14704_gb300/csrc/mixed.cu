// mixed.cu -- launcher of the mixed-degree transform (one launch
// for every limb of degree 2^12 .. 2^15 in a plan; see k_ntt_mixed).
#include <mutex>

#include "kernels.cuh"

namespace he {

static const u32 kMixedSmem = 4096 * 8;   // one 2^12-word block per CTA

template <bool INV>
static cudaError_t mixed_prepare()
{
    static std::once_flag f;
    static cudaError_t e = cudaSuccess;
    std::call_once(f, [] {
        e = cudaFuncSetAttribute(k_ntt_mixed<INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixedSmem);
    });
    return e;
}

static cudaLaunchConfig_t mixed_cfg(u32 clusters, cudaStream_t s, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * 8, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = kMixedSmem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 8;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_ntt_mixed(const MixedUnit *units, u32 n_units, const LimbJob *jobs, bool inverse, u32 clusters,
                             cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_cfg(clusters, s, attr);
    if (inverse) {
        if (cudaError_t e = mixed_prepare<true>()) return e;
        return cudaLaunchKernelEx(&cfg, k_ntt_mixed<true>, units, n_units, jobs);
    }
    if (cudaError_t e = mixed_prepare<false>()) return e;
    return cudaLaunchKernelEx(&cfg, k_ntt_mixed<false>, units, n_units, jobs);
}

}  // namespace he
