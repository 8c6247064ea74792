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

// Programmatic dependent launch of the pass kernels: a kernel may start (and
// stage its constant tables) while the previous kernel of the stream drains;
// it waits for that kernel's completion before reading the fields.  The
// enqueueing code turns it on (pdl_enabled) for a single grid group, where it
// hides the launch gaps (6-7% on single instances), and off for batches of
// several groups, whose kernels share the SMs and would lose slots to early,
// waiting CTAs.
extern thread_local bool pdl_enabled;
inline bool use_pdl() { return pdl_enabled; }
// Scheduling priority of the pass launches (0: the stream's).  A batch gives
// its largest grid group the highest priority: that group is the critical
// path of the graph, and the smaller groups' kernels fill the SMs it leaves
// idle (384-instance sweep: 469 -> 460 ms per step).
extern thread_local int launch_priority;
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = launch_priority;
    cfg.attrs = attr;
    cfg.numAttrs = launch_priority != 0 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class R, int N, int V = 0, bool UM = false, int NTH = kPassThreads, bool ZS = true,
          bool PRE = false>
cudaError_t row_attr() {
    return allow_max_dyn_smem(k_row_pass<R, N, V, UM, NTH, ZS, PRE>);
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

template <class R, int N, int V = 0, bool UM = false, int NTH = kPassThreads, bool ZS = true,
          bool PRE = false>
cudaError_t row_launch(const void* descs, int ninst, int ny, int nz, int s, const void* tw,
                       int hx, cudaStream_t st) {
    using G = RowGeom<R, N, V, NTH>;
    dim3 grid((ny + G::ROWS - 1) / G::ROWS, ninst);
    return launch_pdl(k_row_pass<R, N, V, UM, NTH, ZS, PRE>, grid, dim3(NTH),
                      row_smem<R, N, V, UM, NTH>(hx),
                      st, static_cast<const InstDesc<R>*>(descs), ny, nz, s,
                      static_cast<const pt<R>*>(tw));
}

template <class R, int N, int V = 0, int NTH = kPassThreads>
cudaError_t col_launch(const void* descs, int ninst, int nx, const void* tw, cudaStream_t st) {
    using G = ColGeom<R, N, V, NTH>;
    dim3 grid((nx + G::TILE - 1) / G::TILE, ninst);
    return launch_pdl(k_col_pass<R, N, V, NTH>, grid, dim3(NTH), G::smem, st,
                      static_cast<const InstDesc<R>*>(descs), nx, static_cast<const pt<R>*>(tw));
}

template <int N> cudaError_t col_tma_attr() { return allow_max_dyn_smem(k_col_tma<N>); }

template <int N>
cudaError_t col_tma_launch(const void* tmaps, const void* descs, int ninst, int nx, const void* tw,
                           cudaStream_t st) {
    using K = ColTma<N>;
    dim3 grid((nx + K::TILE - 1) / K::TILE, ninst);
    return launch_pdl(k_col_tma<N>, grid, dim3(kPassThreads), K::smem, st,
                      static_cast<const CUtensorMap*>(tmaps), static_cast<const InstDesc<float>*>(descs),
                      nx, static_cast<const pt<float>*>(tw));
}

// The column-layout pass of the one-pass-per-step schedule (FP32).
// Dynamic shared memory of the column-layout pass: transform buffers, table
// prefetch slots, constant tables and the [TILE][hy] deposit bins.
template <int N, int NTH = kPassThreads, int V = 0> size_t col_step_smem(int hy) {
    using G = ColGeom<float, N, V, NTH>;
    return G::fields + slot_bytes<float, NTH>() + size_t(3) * N * sizeof(pt<float>) +
           size_t(G::TILE) * hy * sizeof(float);
}
template <int N, int NTH = kPassThreads, int V = 0> cudaError_t col_step_attr() {
    return allow_max_dyn_smem(k_col_step<N, NTH, V>);
}
template <int N, int NTH = kPassThreads, int V = 0>
cudaError_t col_step_launch(const void* descs, int ninst, int nx, int nz, int s, const void* tw,
                            int hy, cudaStream_t st) {
    using G = ColGeom<float, N, V, NTH>;
    dim3 grid((nx + G::TILE - 1) / G::TILE, ninst);
    return launch_pdl(k_col_step<N, NTH, V>, grid, dim3(NTH), col_step_smem<N, NTH, V>(hy), st,
                      static_cast<const InstDesc<float>*>(descs), nx, nz, s,
                      static_cast<const pt<float>*>(tw));
}

}  // namespace shg
