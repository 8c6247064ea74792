// Launcher of the cluster-resident single-instance propagation (cluster.cuh).
#include <cstdlib>
#include <mutex>

#include "cluster.cuh"
#include "plan.h"

namespace shg {

template <int N, int K> static cudaLaunchConfig_t cluster_cfg(int ninst, cudaStream_t st,
                                                              cudaLaunchAttribute* attr) {
    using G = ClusterGeom<N, K>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K, ninst, 1);
    cfg.blockDim = dim3(G::NT, 1, 1);
    cfg.dynamicSmemBytes = G::smem;
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
template <int N, int K> static bool cluster_usable() {
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        auto kern = k_cluster_prop<N, K>;
        if (K > 8 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(ClusterGeom<N, K>::smem)) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_cfg<N, K>(1, nullptr, attr);
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
static cudaError_t launch_k(const void* descs, int ninst, int nz, const void* tw, cudaStream_t st) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg<N, K>(ninst, st, attr);
    return cudaLaunchKernelEx(&cfg, k_cluster_prop<N, K>, static_cast<const InstDesc<float>*>(descs),
                              nz, static_cast<const float4*>(tw));
}

// Cluster size used for an N x N instance (0: no cluster path for N).
int cluster_size(int n) {
    if (n == 128) return cluster_usable<128, 16>() ? 16 : (cluster_usable<128, 8>() ? 8 : 0);
    if (n == 64) return cluster_usable<64, 8>() ? 8 : (cluster_usable<64, 4>() ? 4 : 0);
    return 0;
}

bool cluster_path(const std::vector<shg_plan*>& plans) {
    const char* v = getenv("SHG_CLUSTER");
    if (v && v[0] == '0') return false;
    if (plans.size() != 1) return false;
    const shg_plan* p = plans[0];
    if (p->fp64 || p->g.nx != p->g.ny || (p->flags & SHG_FLAG_ADJOINT) || p->mon) return false;
    if ((p->flags & SHG_FLAG_THERMAL) && p->Q) return false;   // no heat deposits here
    if (p->ttab && row_umap_bit(plans) == 0) return false;      // maps only via the per-point table
    return cluster_size(p->g.nx) > 0;
}

cudaError_t launch_cluster(int n, const void* descs, int ninst, int nz, const void* tw,
                           cudaStream_t st) {
    switch (cluster_size(n) * 10000 + n) {
        case 160128: return launch_k<128, 16>(descs, ninst, nz, tw, st);
        case 80128: return launch_k<128, 8>(descs, ninst, nz, tw, st);
        case 80064: return launch_k<64, 8>(descs, ninst, nz, tw, st);
        case 40064: return launch_k<64, 4>(descs, ninst, nz, tw, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace shg
