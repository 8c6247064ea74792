// Single-precision instantiations of the row and column passes (n = 8..1024),
// with the alternative FFT shape (variant 1) for n = 64, 128, 256.
#include "launch_passes.cuh"
#include "plan.h"

namespace shg {

#define SHG_F32_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)
#define SHG_F32_VARIANT_SIZES(X) X(64) X(128) X(256)
#define SHG_F32_TMA_SIZES(X) X(32) X(64) X(128) X(256) X(512) X(1024)
#define SHG_F32_WIDE_SIZES(X) X(512) X(1024)

bool has_variant_f32(int n) { return n == 64 || n == 128 || n == 256; }
bool has_col_small_f32(int n) { return n == 64 || n == 128 || n == 256; }
bool has_col_wide_f32(int n) { return n == 512 || n == 1024; }

// v: flavour (0, 1: FFT shape; 3, 4: shape 0 in 128- or 64-thread CTAs; 5, column
// pass only: shape 0 in 512-thread CTAs at 512 and 1024), plus kRowUmap
// to read the per-point temperature table.
template <bool UM>
static cudaError_t row_f32_um(int nx, int v, const void* descs, int ninst, int ny, int nz, int s,
                              const void* tw, int hx, cudaStream_t st) {
    if (v == 3 || v == 4) {
        switch (nx) {
#define X(n)                                                                               \
    case n:                                                                                \
        return v == 3 ? row_launch<float, n, 0, UM, 128>(descs, ninst, ny, nz, s, tw, hx, st) \
                      : row_launch<float, n, 0, UM, 64>(descs, ninst, ny, nz, s, tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 1) {
        switch (nx) {
#define X(n) case n: return row_launch<float, n, 1, UM>(descs, ninst, ny, nz, s, tw, hx, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    switch (nx) {
#define X(n) case n: return row_launch<float, n, 0, UM>(descs, ninst, ny, nz, s, tw, hx, st);
        SHG_F32_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

// passes_f32_lean.cu: the table-path rows without the code at z_s.
cudaError_t row_f32_lean(int nx, int v, const void* descs, int ninst, int ny, int nz, int s,
                         const void* tw, int hx, cudaStream_t st);
cudaError_t attr_f32_lean();

cudaError_t row_f32(int nx, int v, const void* descs, int ninst, int ny, int nz, int s,
                    const void* tw, int hx, cudaStream_t st) {
    if ((v & kRowUmap) && (v & kRowLean))
        return row_f32_lean(nx, v & ~(kRowUmap | kRowLean), descs, ninst, ny, nz, s, tw, hx, st);
    v &= ~kRowLean;
    return (v & kRowUmap) ? row_f32_um<true>(nx, v & ~kRowUmap, descs, ninst, ny, nz, s, tw, hx, st)
                          : row_f32_um<false>(nx, v, descs, ninst, ny, nz, s, tw, hx, st);
}

// Column tile width of the TMA-staged column pass for length ny (0: none).
int col_tma_tile_f32(int ny) {
    switch (ny) {
#define X(n) case n: return ColTma<n>::TILE;
        SHG_F32_TMA_SIZES(X)
#undef X
    }
    return 0;
}

cudaError_t col_f32(int ny, int v, const void* descs, int ninst, int nx, const void* tw,
                    cudaStream_t st, const void* tmaps) {
    if (v == 2 && tmaps != nullptr) {
        switch (ny) {
#define X(n) case n: return col_tma_launch<n>(tmaps, descs, ninst, nx, tw, st);
            SHG_F32_TMA_SIZES(X)
#undef X
        }
    }
    if (v == 5) {
        switch (ny) {
#define X(n) case n: return col_launch<float, n, 0, 512>(descs, ninst, nx, tw, st);
            SHG_F32_WIDE_SIZES(X)
#undef X
        }
    }
    if (v == 3 || v == 4) {
        switch (ny) {
#define X(n)                                                                  \
    case n:                                                                   \
        return v == 3 ? col_launch<float, n, 0, 128>(descs, ninst, nx, tw, st) \
                      : col_launch<float, n, 0, 64>(descs, ninst, nx, tw, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 1) {
        switch (ny) {
#define X(n) case n: return col_launch<float, n, 1>(descs, ninst, nx, tw, st);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    switch (ny) {
#define X(n) case n: return col_launch<float, n>(descs, ninst, nx, tw, st);
        SHG_F32_SIZES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

// Per-point temperature table: the bilinear sample (dT, C) of map layer l at
// field point (x, y), with the same cell arithmetic as the passes' node
// sampler, stored per adjacent point pair as (dT_2j, dT_2j+1, C_2j, C_2j+1)
// ([tz][ny][nx/2] float4, FP32).  One thread samples both points of pair j
// and writes the entry with one 16-byte store.
SHG_D void upsample_pair(const InstDesc<float>& d, float4* __restrict__ out, int nx, int ny, int j,
                         int y, int l) {
    const MapView<float> mv{d.ttab, d.tx, d.tx * d.ty, 0, 0, 0};
    const RowCell<float> rc = row_cell(d, y);
    TempSampler<float> s0, s1;
    make_sampler(d, mv, 2 * j, rc, s0);
    make_sampler(d, mv, 2 * j + 1, rc, s1);
    const float2 a = s0.bil(l), b = s1.bil(l);
    out[(size_t(l) * ny + y) * (nx / 2) + j] = make_float4(a.x, b.x, a.y, b.y);
}

// grid = (ceil(nx / 2 / kUpsThreads), ny, tz)
constexpr int kUpsThreads = 128;
__global__ void k_upsample_map(const InstDesc<float>* __restrict__ dp, float4* __restrict__ out,
                               int nx, int ny) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nx / 2) upsample_pair(*dp, out, nx, ny, j, blockIdx.y, blockIdx.z);
}

// The same for n plans of one grid: blockIdx.z = plan * tz + layer.
__global__ void k_upsample_map_batch(const InstDesc<float>* const* __restrict__ dps,
                                     float4* const* __restrict__ outs, int nx, int ny, int tz) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.z / tz, l = blockIdx.z - k * tz;
    if (j < nx / 2) upsample_pair(*dps[k], outs[k], nx, ny, j, blockIdx.y, l);
}

cudaError_t launch_upsample_map(const void* desc, void* umap, int nx, int ny, int tz,
                                cudaStream_t st) {
    if (tz > 65535) return cudaErrorInvalidValue;
    dim3 grid((nx / 2 + kUpsThreads - 1) / kUpsThreads, ny, tz);
    k_upsample_map<<<grid, kUpsThreads, 0, st>>>(static_cast<const InstDesc<float>*>(desc),
                                                static_cast<float4*>(umap), nx, ny);
    return cudaGetLastError();
}

cudaError_t launch_upsample_map_batch(const void* const* descs, void* const* umaps, int n, int nx,
                                      int ny, int tz, cudaStream_t st) {
    if (size_t(n) * tz > 65535) return cudaErrorInvalidValue;
    dim3 grid((nx / 2 + kUpsThreads - 1) / kUpsThreads, ny, n * tz);
    k_upsample_map_batch<<<grid, kUpsThreads, 0, st>>>(
        reinterpret_cast<const InstDesc<float>* const*>(descs),
        reinterpret_cast<float4* const*>(umaps), nx, ny, tz);
    return cudaGetLastError();
}

cudaError_t attr_f32() {
    cudaError_t e = cudaSuccess;
#define X(n)                                                    \
    if (e == cudaSuccess) e = row_attr<float, n>();             \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true>();    \
    if (e == cudaSuccess) e = col_attr<float, n>();
    SHG_F32_SIZES(X)
#undef X
#define X(n)                                                     \
    if (e == cudaSuccess) e = row_attr<float, n, 1>();           \
    if (e == cudaSuccess) e = row_attr<float, n, 1, true>();     \
    if (e == cudaSuccess) e = row_attr<float, n, 0, false, 128>(); \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 128>();  \
    if (e == cudaSuccess) e = row_attr<float, n, 0, false, 64>();  \
    if (e == cudaSuccess) e = row_attr<float, n, 0, true, 64>();   \
    if (e == cudaSuccess) e = col_attr<float, n, 1>();           \
    if (e == cudaSuccess) e = col_attr<float, n, 0, 128>();      \
    if (e == cudaSuccess) e = col_attr<float, n, 0, 64>();
    SHG_F32_VARIANT_SIZES(X)
#undef X
#define X(n) \
    if (e == cudaSuccess) e = col_tma_attr<n>();
    SHG_F32_TMA_SIZES(X)
#undef X
#define X(n) \
    if (e == cudaSuccess) e = col_attr<float, n, 0, 512>();
    SHG_F32_WIDE_SIZES(X)
#undef X
    if (e == cudaSuccess) e = attr_f32_lean();
    return e;
}

size_t row_smem_f32(int nx, int v, int hx) {
    const bool um = (v & kRowUmap) != 0;
    v &= ~(kRowUmap | kRowLean);
    if (v == 3) {
        switch (nx) {
#define X(n) case n: return um ? row_smem<float, n, 0, true, 128>(hx) : row_smem<float, n, 0, false, 128>(hx);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 4) {
        switch (nx) {
#define X(n) case n: return um ? row_smem<float, n, 0, true, 64>(hx) : row_smem<float, n, 0, false, 64>(hx);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    if (v == 1) {
        switch (nx) {
#define X(n) case n: return um ? row_smem<float, n, 1, true>(hx) : row_smem<float, n, 1>(hx);
            SHG_F32_VARIANT_SIZES(X)
#undef X
        }
    }
    switch (nx) {
#define X(n) case n: return um ? row_smem<float, n, 0, true>(hx) : row_smem<float, n>(hx);
        SHG_F32_SIZES(X)
#undef X
    }
    return 0;
}

}  // namespace shg
