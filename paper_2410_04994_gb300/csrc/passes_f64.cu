// Double-precision instantiations of the row and column passes (n = 8..256).
#include "launch_passes.cuh"
#include "plan.h"

namespace shg {

#define SHG_F64_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256)

cudaError_t row_f64(int nx, int, const void* descs, int ninst, int ny, int nz, int s,
                    const void* tw, int hx, cudaStream_t st) {
    switch (nx) {
#define X(n) case n: return row_launch<double, n>(descs, ninst, ny, nz, s, tw, hx, st);
        SHG_F64_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t col_f64(int ny, int, const void* descs, int ninst, int nx, const void* tw,
                    cudaStream_t st, const void*) {
    switch (ny) {
#define X(n) case n: return col_launch<double, n>(descs, ninst, nx, tw, st);
        SHG_F64_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t attr_f64() {
    cudaError_t e = cudaSuccess;
#define X(n)                                        \
    if (e == cudaSuccess) e = row_attr<double, n>(); \
    if (e == cudaSuccess) e = col_attr<double, n>();
    SHG_F64_SIZES(X)
#undef X
    return e;
}

size_t row_smem_f64(int nx, int, int hx) {
    switch (nx) {
#define X(n) case n: return row_smem<double, n>(hx);
        SHG_F64_SIZES(X)
#undef X
    }
    return 0;
}

}  // namespace shg
