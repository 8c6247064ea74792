// Single-precision passes of the one-pass-per-step schedule: the row-layout
// pass (k_row_pass with the per-point table, without the z_s code, with Lx
// before the nonlinear part) in every flavour of the monitor-free rows, and
// the column-layout pass k_col_step (n = 8..1024).  A translation unit of its
// own so that the library builds in parallel.
#include "launch_passes.cuh"
#include "plan.h"

namespace shg {

#define SHG_F32_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)
#define SHG_F32_VARIANT_SIZES(X) X(64) X(128) X(256)
#define SHG_F32_SMALL_COL_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512)

bool has_col_step_small_f32(int n) { return n >= 8 && n <= 512; }
bool has_col_step_wide_f32(int n) { return n == 512 || n == 1024; }
bool has_col_step_v1_f32(int n) { return n == 64 || n == 128 || n == 256; }

// v: the row flavour (0, 1, 3, 4) without the row-pass bits.
cudaError_t row_f32_step(int nx, int v, const void* descs, int ninst, int ny, int nz, int s,
                         const void* tw, int hx, cudaStream_t st) {
    if (v == 3 || v == 4) {
        switch (nx) {
#define X(n)                                                                                   \
    case n:                                                                                    \
        return v == 3 ? row_launch<float, n, 0, true, 128, false, true>(descs, ninst, ny, nz, s, \
                                                                         tw, hx, st)            \
                      : row_launch<float, n, 0, true, 64, false, true>(descs, ninst, ny, nz, s,  \
                                                                        tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 1) {
        switch (nx) {
#define X(n)                                                                                   \
    case n:                                                                                    \
        return row_launch<float, n, 1, true, kPassThreads, false, true>(descs, ninst, ny, nz, s, \
                                                                         tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    switch (nx) {
#define X(n)                                                                                   \
    case n:                                                                                    \
        return row_launch<float, n, 0, true, kPassThreads, false, true>(descs, ninst, ny, nz, s, \
                                                                         tw, hx, st);
        SHG_F32_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

// v: 3 for 128-thread CTAs (lengths up to 512: half the columns per CTA), 5
// for 512-thread CTAs (lengths 512 and 1024: twice the columns, so that a
// warp reads whole 32-byte sectors of each row), 1 for the 8-element shape in
// 256-thread CTAs (lengths 64 to 256: three CTAs per SM), else the 16-element
// shape in 256-thread CTAs.
cudaError_t col_f32_step(int ny, int v, const void* descs, int ninst, int nx, int nz, int s,
                         const void* tw, int hy, cudaStream_t st) {
    if (v == 1) {
        switch (ny) {
#define X(n) case n: return col_step_launch<n, kPassThreads, 1>(descs, ninst, nx, nz, s, tw, hy, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 5) {
        switch (ny) {
            case 512: return col_step_launch<512, 512>(descs, ninst, nx, nz, s, tw, hy, st);
            case 1024: return col_step_launch<1024, 512>(descs, ninst, nx, nz, s, tw, hy, st);
        }
    }
    if (v == 3) {
        switch (ny) {
#define X(n) case n: return col_step_launch<n, 128>(descs, ninst, nx, nz, s, tw, hy, st);
            SHG_F32_SMALL_COL_SIZES(X)
#undef X
        }
    }
    switch (ny) {
#define X(n) case n: return col_step_launch<n>(descs, ninst, nx, nz, s, tw, hy, st);
        SHG_F32_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t attr_f32_step() {
    cudaError_t e = cudaSuccess;
#define X(n)                                                                           \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, kPassThreads, false, true>(); \
    if (e == cudaSuccess) e = col_step_attr<n>();
    SHG_F32_SIZES(X)
#undef X
#define X(n) \
    if (e == cudaSuccess) e = col_step_attr<n, 128>();
    SHG_F32_SMALL_COL_SIZES(X)
#undef X
    if (e == cudaSuccess) e = col_step_attr<512, 512>();
    if (e == cudaSuccess) e = col_step_attr<1024, 512>();
#define X(n) \
    if (e == cudaSuccess) e = col_step_attr<n, kPassThreads, 1>();
    SHG_F32_VARIANT_SIZES(X)
#undef X
#define X(n)                                                                           \
    if (e == cudaSuccess) e = row_attr<float, n, 1, true, kPassThreads, false, true>(); \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 128, false, true>();          \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 64, false, true>();
    SHG_F32_VARIANT_SIZES(X)
#undef X
    return e;
}

}  // namespace shg
