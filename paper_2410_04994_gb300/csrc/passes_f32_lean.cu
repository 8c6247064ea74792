// Single-precision row passes on the per-point temperature table without the
// power monitor's code: the instantiations for groups without a monitor, in
// a translation unit of their own so that the library builds in parallel.
#include "launch_passes.cuh"
#include "plan.h"

namespace shg {

#define SHG_F32_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)
#define SHG_F32_VARIANT_SIZES(X) X(64) X(128) X(256)

cudaError_t row_f32_lean(int nx, int v, const void* descs, int ninst, int ny, int nz, int s,
                         const void* tw, int hx, cudaStream_t st) {
    if (v == 3 || v == 4) {
        switch (nx) {
#define X(n)                                                                                    \
    case n:                                                                                     \
        return v == 3 ? row_launch<float, n, 0, true, 128, false>(descs, ninst, ny, nz, s, tw, hx, st) \
                      : row_launch<float, n, 0, true, 64, false>(descs, ninst, ny, nz, s, tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 1) {
        switch (nx) {
#define X(n) \
    case n: return row_launch<float, n, 1, true, kPassThreads, false>(descs, ninst, ny, nz, s, tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    switch (nx) {
#define X(n) \
    case n: return row_launch<float, n, 0, true, kPassThreads, false>(descs, ninst, ny, nz, s, tw, hx, st);
        SHG_F32_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t attr_f32_lean() {
    cudaError_t e = cudaSuccess;
#define X(n) \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, kPassThreads, false>();
    SHG_F32_SIZES(X)
#undef X
#define X(n)                                                                 \
    if (e == cudaSuccess) e = row_attr<float, n, 1, true, kPassThreads, false>(); \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 128, false>();      \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 64, false>();
    SHG_F32_VARIANT_SIZES(X)
#undef X
    return e;
}

}  // namespace shg
