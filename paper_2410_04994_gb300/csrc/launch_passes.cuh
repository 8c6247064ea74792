// Template launchers of the two pass kernels for one precision.
#pragma once
#include "passes.cuh"

namespace shg {

// Largest dynamic shared memory a kernel may request: the device's opt-in
// per-block limit minus the kernel's static shared memory.
template <class K> cudaError_t allow_max_dyn_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - int(a.sharedSizeBytes));
    return e;
}

template <class R, int N, int V = 0, bool UM = false, int NTH = kPassThreads>
cudaError_t row_attr() {
    return allow_max_dyn_smem(k_row_pass<R, N, V, UM, NTH>);
}

// Dynamic shared memory of a row pass: transform buffers + table prefetch
// slots (UM) + deposit bins.
template <class R, int N, int V = 0, bool UM = false, int NTH = kPassThreads>
size_t row_smem(int hx) {
    using G = RowGeom<R, N, V, NTH>;
    return G::fields + (UM ? slot_bytes<R, NTH>() : 0) + G::tables + size_t(G::ROWS) * hx * sizeof(float);
}
template <class R, int N, int V = 0, int NTH = kPassThreads> cudaError_t col_attr() {
    return allow_max_dyn_smem(k_col_pass<R, N, V, NTH>);
}

template <class R, int N, int V = 0, bool UM = false, int NTH = kPassThreads>
cudaError_t row_launch(const void* descs, int ninst, int ny, int nz, int s, const void* tw,
                       int hx, cudaStream_t st) {
    using G = RowGeom<R, N, V, NTH>;
    dim3 grid((ny + G::ROWS - 1) / G::ROWS, ninst);
    k_row_pass<R, N, V, UM, NTH><<<grid, NTH, row_smem<R, N, V, UM, NTH>(hx), st>>>(
        static_cast<const InstDesc<R>*>(descs), ny, nz, s, static_cast<const pt<R>*>(tw));
    return cudaGetLastError();
}

template <class R, int N, int V = 0, int NTH = kPassThreads>
cudaError_t col_launch(const void* descs, int ninst, int nx, const void* tw, cudaStream_t st) {
    using G = ColGeom<R, N, V, NTH>;
    dim3 grid((nx + G::TILE - 1) / G::TILE, ninst);
    k_col_pass<R, N, V, NTH><<<grid, NTH, G::smem, st>>>(static_cast<const InstDesc<R>*>(descs),
                                                          nx, static_cast<const pt<R>*>(tw));
    return cudaGetLastError();
}

template <int N> cudaError_t col_tma_attr() { return allow_max_dyn_smem(k_col_tma<N>); }

template <int N>
cudaError_t col_tma_launch(const void* tmaps, const void* descs, int ninst, int nx, const void* tw,
                           cudaStream_t st) {
    using K = ColTma<N>;
    dim3 grid((nx + K::TILE - 1) / K::TILE, ninst);
    k_col_tma<N><<<grid, kPassThreads, K::smem, st>>>(static_cast<const CUtensorMap*>(tmaps),
                                                      static_cast<const InstDesc<float>*>(descs),
                                                      nx, static_cast<const pt<float>*>(tw));
    return cudaGetLastError();
}

}  // namespace shg
