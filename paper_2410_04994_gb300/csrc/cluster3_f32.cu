// Launcher of the cluster-resident three-wave propagation (cluster3.cuh).
#include <cstdlib>
#include <mutex>

#include "cluster3.cuh"
#include "plan.h"

namespace shg {

template <int N, int K> static cudaLaunchConfig_t cluster3_cfg(cudaStream_t st,
                                                               cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K, 1, 1);
    cfg.blockDim = dim3(Cluster3Geom<N, K>::NT, 1, 1);
    cfg.dynamicSmemBytes = Cluster3Geom<N, K>::smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Attributes once per kernel, and whether one cluster of it can be resident.
template <int N, int K> static bool cluster3_usable() {
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        auto kern = k_cluster3<N, K>;
        if (K > 8 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Cluster3Geom<N, K>::smem)) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster3_cfg<N, K>(nullptr, attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        ok = n > 0;
    });
    return ok;
}

template <int N, int K>
static cudaError_t launch3_k(const void* q, int nz, const void* tw, cudaStream_t st) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster3_cfg<N, K>(st, attr);
    return cudaLaunchKernelEx(&cfg, k_cluster3<N, K>, static_cast<const Inst3<float>*>(q), nz,
                              static_cast<const float4*>(tw));
}

// Cluster size for an N x N three-wave instance (0: no cluster path for N).
// 128: 16 CTAs of 384 threads (8 rows each); 64: 8 CTAs of 192 threads, or 4
// of 384.
int cluster3_size(int n) {
    if (n == 128) return cluster3_usable<128, 16>() ? 16 : 0;
    if (n == 64) return cluster3_usable<64, 8>() ? 8 : (cluster3_usable<64, 4>() ? 4 : 0);
    return 0;
}

bool cluster3_path(const shg_plan* p) {
    const char* v = getenv("SHG_CLUSTER");
    if (v && v[0] == '0') return false;
    if (p->fp64 || p->g.nx != p->g.ny) return false;
    // maps only via the per-point table, whose layers one step may not outrun
    if (p->ttab && (!p->umap || !(double(p->tz - 1) < 0.99 * p->g.nz))) return false;
    return cluster3_size(p->g.nx) > 0;
}

cudaError_t launch_cluster3(int n, const void* q, int nz, const void* tw, cudaStream_t st) {
    switch (cluster3_size(n) * 10000 + n) {
        case 160128: return launch3_k<128, 16>(q, nz, tw, st);
        case 80064: return launch3_k<64, 8>(q, nz, tw, st);
        case 40064: return launch3_k<64, 4>(q, nz, tw, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace shg
