// Template launchers of the two pass kernels for one precision.
#pragma once
#include "passes.cuh"

namespace shg {

template <class R, int N> cudaError_t row_attr() {
    return cudaFuncSetAttribute(k_row_pass<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(RowGeom<R, N>::smem));
}
template <class R, int N> cudaError_t col_attr() {
    return cudaFuncSetAttribute(k_col_pass<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(ColGeom<R, N>::smem));
}

template <class R, int N>
cudaError_t row_launch(const void* descs, int ninst, int ny, int nz, int s, const void* tw,
                       cudaStream_t st) {
    using G = RowGeom<R, N>;
    dim3 grid((ny + G::ROWS - 1) / G::ROWS, ninst);
    k_row_pass<R, N><<<grid, kPassThreads, G::smem, st>>>(
        static_cast<const InstDesc<R>*>(descs), ny, nz, s, static_cast<const pt<R>*>(tw));
    return cudaGetLastError();
}

template <class R, int N>
cudaError_t col_launch(const void* descs, int ninst, int nx, const void* tw, cudaStream_t st) {
    using G = ColGeom<R, N>;
    dim3 grid((nx + G::TILE - 1) / G::TILE, ninst);
    k_col_pass<R, N><<<grid, kPassThreads, G::smem, st>>>(static_cast<const InstDesc<R>*>(descs),
                                                          nx, static_cast<const pt<R>*>(tw));
    return cudaGetLastError();
}

}  // namespace shg
