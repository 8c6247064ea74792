// Single-precision instantiations of the transposed row pass.
#include "adjoint_pass.cuh"
#include "launch_passes.cuh"

namespace shg {

// The adjoint sweep runs one instance, so its row kernel uses small CTAs
// (NTH = max(64, T) threads, a few rows each) to spread the rows over more SMs.
template <class R, int N>
static cudaError_t row_adj_launch(const void* dl, const void* Y, AdjAcc acc, int ny, int nz,
                                  int s, const void* tw, cudaStream_t st) {
    constexpr int T = FftCfg<R, N>::T, NTH = T > 64 ? T : 64;
    using G = RowGeom<R, N, 0, NTH>;
    static const cudaError_t attr = allow_max_dyn_smem(k_row_adj<R, N, NTH>);  // once, thread-safe
    if (attr != cudaSuccess) return attr;
    dim3 grid((ny + G::ROWS - 1) / G::ROWS, 1);
    k_row_adj<R, N, NTH><<<grid, NTH, G::fields + G::tables, st>>>(
        static_cast<const InstDesc<R>*>(dl), static_cast<const cx<R>*>(Y), acc, ny, nz, s,
        static_cast<const pt<R>*>(tw));
    return cudaGetLastError();
}

cudaError_t row_adj_f32(int nx, const void* dl, const void* Y, AdjAcc acc, int ny, int nz, int s,
                        const void* tw, cudaStream_t st) {
    switch (nx) {
#define X(n) case n: return row_adj_launch<float, n>(dl, Y, acc, ny, nz, s, tw, st);
        X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace shg
