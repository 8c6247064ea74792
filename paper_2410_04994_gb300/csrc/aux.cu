// Initial pump, FP64 power reductions and temperature tables.
#include "plan.h"

namespace shg {

cudaError_t row_f32(int, int, const void*, int, int, int, int, const void*, int, cudaStream_t);
cudaError_t row_f64(int, int, const void*, int, int, int, int, const void*, int, cudaStream_t);
size_t row_smem_f32(int, int, int);
size_t row_smem_f64(int, int, int);
cudaError_t col_f32(int, int, const void*, int, int, const void*, cudaStream_t, const void*);
cudaError_t col_f64(int, int, const void*, int, int, const void*, cudaStream_t, const void*);
int col_tma_tile_f32(int);
bool has_variant_f32(int);
bool has_col_small_f32(int);
bool has_col_wide_f32(int);
cudaError_t attr_f32();
cudaError_t attr_f64();
cudaError_t row_f32_step(int, int, const void*, int, int, int, int, const void*, int, cudaStream_t);
cudaError_t col_f32_step(int, int, const void*, int, int, int, int, const void*, int, cudaStream_t);
bool has_col_step_small_f32(int);
bool has_col_step_wide_f32(int);
bool has_col_step_v1_f32(int);
cudaError_t attr_f32_step();

thread_local bool pdl_enabled = false;
thread_local int launch_priority = 0;

bool has_fft_variant(bool fp64, int n) { return !fp64 && has_variant_f32(n); }
bool has_col_small(bool fp64, int n) { return !fp64 && has_col_small_f32(n); }
bool has_col_wide(bool fp64, int n) { return !fp64 && has_col_wide_f32(n); }

cudaError_t launch_row(bool fp64, int nx, const void* descs, int ninst, int ny, int nz, int s,
                       const void* tw, int hx, cudaStream_t st, int variant) {
    return fp64 ? row_f64(nx, variant, descs, ninst, ny, nz, s, tw, hx, st)
                : row_f32(nx, variant, descs, ninst, ny, nz, s, tw, hx, st);
}

size_t row_pass_smem(bool fp64, int nx, int hx, int variant) {
    return fp64 ? row_smem_f64(nx, variant, hx) : row_smem_f32(nx, variant, hx);
}

cudaError_t launch_col(bool fp64, int ny, const void* descs, int ninst, int nx, const void* tw,
                       cudaStream_t st, int variant, const void* tmaps) {
    return fp64 ? col_f64(ny, variant, descs, ninst, nx, tw, st, tmaps)
                : col_f32(ny, variant, descs, ninst, nx, tw, st, tmaps);
}

int col_tma_tile(bool fp64, int ny) { return fp64 ? 0 : col_tma_tile_f32(ny); }

cudaError_t launch_row_step(int nx, const void* descs, int ninst, int ny, int nz, int s,
                            const void* tw, int hx, cudaStream_t st, int variant) {
    return row_f32_step(nx, variant & ~(kRowUmap | kRowLean), descs, ninst, ny, nz, s, tw, hx, st);
}

cudaError_t launch_col_step(int ny, const void* descs, int ninst, int nx, int nz, int s,
                            const void* tw, int hy, cudaStream_t st, int variant) {
    return col_f32_step(ny, variant, descs, ninst, nx, nz, s, tw, hy, st);
}

bool has_col_step_small(int n) { return has_col_step_small_f32(n); }
bool has_col_step_wide(int n) { return has_col_step_wide_f32(n); }
bool has_col_step_v1(int n) { return has_col_step_v1_f32(n); }

cudaError_t setup_pass_attributes() {
    cudaError_t e = attr_f32();
    if (e == cudaSuccess) e = attr_f64();
    if (e == cudaSuccess) e = attr_f32_step();
    return e;
}

constexpr int kRedThreads = 256;

// Block-wide sum of two doubles in a fixed order (deterministic).
__device__ void block_sum2(double& a, double& b) {
    __shared__ double sa[kRedThreads], sb[kRedThreads];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    a = sa[0];
    b = sb[0];
    __syncthreads();
}

// Unnormalised Eq. (5) at z = 0: exp(-r^2 / (w0^2 (1 + i tau0))) / (1 + i tau0),
// tau0 = -z_focus / z_R, z_R = w0^2 k_F / 2 (double precision).
__device__ double2 gauss0(const InitDesc& d, int m, int n) {
    const double x = d.x0 + d.dx * m, y = d.y0 + d.dy * n;
    const double zr = d.w0 * d.w0 * d.kF * 0.5;
    const double tau = -d.zf / zr;
    // 1/(1 + i tau) = (1 - i tau) / (1 + tau^2)
    const double den = 1.0 + tau * tau;
    const double qr = 1.0 / den, qi = -tau / den;
    const double a = -(x * x + y * y) / (d.w0 * d.w0);  // exponent = a * (qr + i qi)
    const double mag = exp(a * qr);
    double s, c;
    sincos(a * qi, &s, &c);
    const double er = mag * c, ei = mag * s;
    return make_double2(er * qr - ei * qi, er * qi + ei * qr);
}

// Pass 1 of the init: partial sums of |g|^2 (or of the custom field power).
__global__ void k_init_partial(const InitDesc* __restrict__ ids, int nx, int ny) {
    const InitDesc& d = ids[blockIdx.y];
    double acc = 0, unused = 0;
    const int npts = nx * ny;
    for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < npts; i += gridDim.x * kRedThreads) {
        double2 g = gauss0(d, i % nx, i / nx);
        acc += g.x * g.x + g.y * g.y;
    }
    block_sum2(acc, unused);
    if (threadIdx.x == 0) d.red[blockIdx.x * 2] = acc;
}

// Pass 2: every block sums the partials in the same order, scales and writes.
template <class R>
__global__ void k_init_write(const InitDesc* __restrict__ ids, const InstDesc<R>* __restrict__ ds,
                             int nx, int ny) {
    using C = cx<R>;
    const InitDesc& d = ids[blockIdx.y];
    C* f = ds[blockIdx.y].field;
    const int npts = nx * ny;
    __shared__ double a0s;
    if (threadIdx.x == 0) {
        double s = 0;
        for (int b = 0; b < kRedBlocks; ++b) s += d.red[b * 2];
        a0s = sqrt(d.p1 / (d.cFdxdy * s));
    }
    __syncthreads();
    const double a0 = a0s;
    for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < npts; i += gridDim.x * kRedThreads) {
        double2 g = gauss0(d, i % nx, i / nx);
        f[i] = mk<C>(R(a0 * g.x), R(a0 * g.y));
        f[npts + i] = mk<C>(R(0), R(0));
    }
}

// Custom initial state: plain copy.
template <class R>
__global__ void k_copy_init(const InitDesc* __restrict__ ids, const InstDesc<R>* __restrict__ ds,
                            int nx, int ny) {
    using C = cx<R>;
    const C* src = static_cast<const C*>(ids[blockIdx.y].f0);
    C* f = ds[blockIdx.y].field;
    const int n2 = 2 * nx * ny;
    for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < n2; i += gridDim.x * kRedThreads)
        f[i] = src[i];
}

cudaError_t launch_init(bool fp64, const InitDesc* idescs, void* const*, int ninst,
                        const void* descs, int nx, int ny, cudaStream_t st) {
    // Instances of one batch either all use the Gaussian or carry f0; the
    // host splits mixed batches.
    dim3 grid(kRedBlocks, ninst);
    k_init_partial<<<grid, kRedThreads, 0, st>>>(idescs, nx, ny);
    if (fp64)
        k_init_write<double><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<double>*>(descs), nx, ny);
    else
        k_init_write<float><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<float>*>(descs), nx, ny);
    return cudaGetLastError();
}

cudaError_t launch_copy_init(bool fp64, const InitDesc* idescs, int ninst, const void* descs,
                             int nx, int ny, cudaStream_t st) {
    dim3 grid(kRedBlocks, ninst);
    if (fp64)
        k_copy_init<double><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<double>*>(descs), nx, ny);
    else
        k_copy_init<float><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<float>*>(descs), nx, ny);
    return cudaGetLastError();
}

// P_j = (1/2) eps0 c n_j sum |A_j|^2 dx dy, summed in double in a fixed order.
template <class R>
__global__ void k_power_partial(const InitDesc* __restrict__ ids,
                                const InstDesc<R>* __restrict__ ds, int nx, int ny) {
    using C = cx<R>;
    const InitDesc& d = ids[blockIdx.y];
    const C* f = ds[blockIdx.y].field;
    const int npts = nx * ny;
    double aF = 0, aS = 0;
    for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < npts; i += gridDim.x * kRedThreads) {
        C u = f[i], v = f[npts + i];
        aF += double(u.x) * u.x + double(u.y) * u.y;
        aS += double(v.x) * v.x + double(v.y) * v.y;
    }
    block_sum2(aF, aS);
    if (threadIdx.x == 0) {
        d.red[blockIdx.x * 2] = aF;
        d.red[blockIdx.x * 2 + 1] = aS;
    }
}

__global__ void k_power_final(const InitDesc* __restrict__ ids) {
    const InitDesc& d = ids[blockIdx.x];
    if (threadIdx.x == 0) {
        double aF = 0, aS = 0;
        for (int b = 0; b < kRedBlocks; ++b) {
            aF += d.red[b * 2];
            aS += d.red[b * 2 + 1];
        }
        d.pw[0] = d.cFdxdy * aF;
        d.pw[1] = d.cSdxdy * aS;
    }
}

cudaError_t launch_power(bool fp64, const InitDesc* idescs, const void* descs, int ninst, int nx,
                         int ny, cudaStream_t st) {
    dim3 grid(kRedBlocks, ninst);
    if (fp64)
        k_power_partial<double><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<double>*>(descs), nx, ny);
    else
        k_power_partial<float><<<grid, kRedThreads, 0, st>>>(
            idescs, static_cast<const InstDesc<float>*>(descs), nx, ny);
    k_power_final<<<ninst, 32, 0, st>>>(idescs);
    return cudaGetLastError();
}

// (dT, C) table: C[l] = C[l-1] + dZ/2 (f[l-1] + f[l]) accumulated in double
// (Eq. 3 by the trapezoid rule on the map's z-nodes) of the integrand f of
// the phase model (dT itself, or Dk(T_ref + dT) - Dk(T_ref) of Eq. 4),
// stored in the plan's precision.
template <class V>
__global__ void k_build_ttab(const float* __restrict__ dT, V* __restrict__ tt, int tx, int ty,
                             int tz, double dZ, DkModel m) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= tx * ty) return;
    const size_t plane = size_t(tx) * ty;
    double c = 0;
    float prev = dT[col];
    double fprev = phase_integrand(m, prev);
    tt[col] = mk<V>(prev, 0);
    // layers in chunks of 16: the loads of a chunk are independent and in
    // flight together; the sum runs in layer order
    constexpr int K = 16;
    for (int l0 = 1; l0 < tz; l0 += K) {
        float cur[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (l0 + k < tz) cur[k] = dT[(l0 + k) * plane + col];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (l0 + k < tz) {
                const double f = phase_integrand(m, cur[k]);
                c += 0.5 * dZ * (fprev + f);
                tt[(l0 + k) * plane + col] = mk<V>(cur[k], c);
                fprev = f;
            }
        }
    }
}

// The same for many maps of one shape at once: job k (blockIdx.y) builds
// jobs[k].tt from jobs[k].src and keeps a copy of the map in jobs[k].copy.
template <class V>
__global__ void k_build_ttab_batch(const TtabJob* __restrict__ jobs, int tx, int ty, int tz) {
    const TtabJob j = jobs[blockIdx.y];
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= tx * ty) return;
    const size_t plane = size_t(tx) * ty;
    V* tt = static_cast<V*>(j.tt);
    double c = 0;
    float prev = j.src[col];
    double fprev = phase_integrand(j.dkm, prev);
    j.copy[col] = prev;
    tt[col] = mk<V>(prev, 0);
    constexpr int K = 16;
    for (int l0 = 1; l0 < tz; l0 += K) {
        float cur[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (l0 + k < tz) cur[k] = j.src[(l0 + k) * plane + col];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (l0 + k < tz) {
                const double f = phase_integrand(j.dkm, cur[k]);
                c += 0.5 * j.dZ * (fprev + f);
                tt[(l0 + k) * plane + col] = mk<V>(cur[k], c);
                j.copy[(l0 + k) * plane + col] = cur[k];
                fprev = f;
            }
        }
    }
}

cudaError_t launch_build_ttab_batch(bool fp64, const TtabJob* jobs, int njobs, int tx, int ty,
                                    int tz, cudaStream_t st) {
    dim3 grid((tx * ty + 127) / 128, njobs);
    if (fp64)
        k_build_ttab_batch<double2><<<grid, 128, 0, st>>>(jobs, tx, ty, tz);
    else
        k_build_ttab_batch<float2><<<grid, 128, 0, st>>>(jobs, tx, ty, tz);
    return cudaGetLastError();
}

cudaError_t launch_build_ttab(bool fp64, const float* dT, void* ttab, int tx, int ty, int tz,
                              double dZ, const DkModel& dkm, cudaStream_t st) {
    const int cols = tx * ty;
    if (fp64)
        k_build_ttab<double2><<<(cols + 127) / 128, 128, 0, st>>>(dT, static_cast<double2*>(ttab),
                                                                   tx, ty, tz, dZ, dkm);
    else
        k_build_ttab<float2><<<(cols + 127) / 128, 128, 0, st>>>(dT, static_cast<float2*>(ttab),
                                                                  tx, ty, tz, dZ, dkm);
    return cudaGetLastError();
}

}  // namespace shg
