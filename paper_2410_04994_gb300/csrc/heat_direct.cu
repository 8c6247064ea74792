// Direct solve of the discrete steady heat equation (Eq. 16) by separation of
// variables, with mixed-precision iterative refinement.
//
// With each face of the crystal either held at the oven temperature (Eq. 9)
// or convective (Eq. 10, ghost-node form), the 7-point operator acting on
// the unknown nodes is a Kronecker sum A = Ax (+) Ay (+) Az of three 1-D
// operators.  Ax and Ay are diagonalised once on the host (their
// symmetrised forms by cyclic Jacobi rotations); then A e = -r is solved by
//   r^ = (Vy^-1 (x) Vx^-1) r           two dense transforms (FP32 GEMMs)
//   (Az + (lx + ly) I) e^ = -r^        one tridiagonal solve per (kx, ky)
//   e  = (Vy (x) Vx) e^                two dense transforms
// and the FP64 temperature is refined, T += e, from the FP64 residual r of
// the node equations until the largest Jacobi correction |r_i| / D_i (the
// stopping test of the SOR as well) is below the tolerance.  Each pass of
// the FP32 solve reduces the error by about six orders, so two or three
// passes reach FP64 rounding; the SOR needs hundreds of FP64 sweeps.
//
// Layout: the unknown nodes of each axis are lo_d .. hi_d (an oven face's
// nodes are excluded), m_d of them; work arrays are [mz][my][mx] float.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.h"

namespace shg {

// ----------------------------------------------------------- host eigen ----

// Eigen-decomposition of the symmetric n x n matrix a (row-major, overwritten)
// by cyclic Jacobi rotations: a = U diag(w) U^T, U column k the k-th vector.
static void jacobi_eig(int n, std::vector<double>& a, std::vector<double>& w,
                       std::vector<double>& U) {
    U.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) U[size_t(i) * n + i] = 1.0;
    auto A = [&](int i, int j) -> double& { return a[size_t(i) * n + j]; };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, diag = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) (i == j ? diag : off) += A(i, j) * A(i, j);
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A(p, q);
                if (std::fabs(apq) <= 1e-300) continue;
                // rotation in the (p, q) plane that zeroes a_pq
                const double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double ukp = U[size_t(k) * n + p], ukq = U[size_t(k) * n + q];
                    U[size_t(k) * n + p] = c * ukp - s * ukq;
                    U[size_t(k) * n + q] = s * ukp + c * ukq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A(i, i);
}

// Unknown range of one axis of n nodes and the ghost-node coefficient of its
// two ends (0 for an oven face, whose nodes are excluded).
struct Axis {
    int n, lo, hi, m;
    double a;           // 1 / d^2
    double add_lo, add_hi;  // 2 a d h / kappa at a convective end, else 0
};

static Axis make_axis(int n, double d, bool conv_lo, bool conv_hi, double h_lo, double h_hi,
                      double kappa) {
    Axis ax;
    ax.n = n;
    ax.lo = conv_lo ? 0 : 1;
    ax.hi = conv_hi ? n - 1 : n - 2;
    ax.m = ax.hi - ax.lo + 1;
    ax.a = 1.0 / (d * d);
    ax.add_lo = conv_lo ? 2.0 * ax.a * d * h_lo / kappa : 0.0;
    ax.add_hi = conv_hi ? 2.0 * ax.a * d * h_hi / kappa : 0.0;
    return ax;
}

// The 1-D operator of an axis on its unknowns (a_d (T_-1 + T_+1 - 2 T), an oven
// neighbour contributing 0, a convective end with its ghost node: 2 a T_inner
// - (2 a + add) T), symmetrised by the half weights of the convective end
// rows, diagonalised: A_d = V diag(lam) V^-1 with V = W^-1/2 U, V^-1 = U^T W^1/2.
static void axis_eigen(const Axis& ax, std::vector<double>& lam, std::vector<double>& V,
                       std::vector<double>& Vinv) {
    const int m = ax.m;
    std::vector<double> A(size_t(m) * m, 0.0), wgt(m, 1.0);
    for (int r = 0; r < m; ++r) {
        const int i = ax.lo + r;
        double diag = -2.0 * ax.a;
        if (i == 0) diag -= ax.add_lo;
        if (i == ax.n - 1) diag -= ax.add_hi;
        A[size_t(r) * m + r] = diag;
        if (r > 0) A[size_t(r) * m + r - 1] = (i == ax.n - 1) ? 2.0 * ax.a : ax.a;
        if (r < m - 1) A[size_t(r) * m + r + 1] = (i == 0) ? 2.0 * ax.a : ax.a;
        if (i == 0 || i == ax.n - 1) wgt[r] = 0.5;
    }
    // W A is symmetric: S = W^1/2 A W^-1/2
    std::vector<double> S(size_t(m) * m);
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c)
            S[size_t(r) * m + c] = std::sqrt(wgt[r]) * A[size_t(r) * m + c] / std::sqrt(wgt[c]);
    for (int r = 0; r < m; ++r)  // remove the rounding asymmetry
        for (int c = r + 1; c < m; ++c) {
            const double v = 0.5 * (S[size_t(r) * m + c] + S[size_t(c) * m + r]);
            S[size_t(r) * m + c] = S[size_t(c) * m + r] = v;
        }
    std::vector<double> U;
    jacobi_eig(m, S, lam, U);
    V.assign(size_t(m) * m, 0.0);
    Vinv.assign(size_t(m) * m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) {
            V[size_t(i) * m + k] = U[size_t(i) * m + k] / std::sqrt(wgt[i]);
            Vinv[size_t(k) * m + i] = U[size_t(i) * m + k] * std::sqrt(wgt[i]);
        }
}

// ------------------------------------------------------------- kernels ----

struct DirGeom {
    int hx, hy, hz;
    int lox, loy, loz, mx, my, mz;
    double ax, ay, az;
    double add[6];      // ghost coefficient of each face (x-, x+, y-, y+, z-, z+), 0 for oven
    double tinf;        // T_inf - T_oven
    double qs;          // 1 / (kappa dx dy dz)
};

// FP64 residual of every unknown node's equation, its Jacobi correction
// (max |res| / D into *maxcorr) and the residual compacted to float [mz][my][mx].
// grid = (ceil(mx / 128), my, mz).
__global__ void k_dir_residual(const double* __restrict__ T, const double* __restrict__ Q,
                               DirGeom g, float* __restrict__ out,
                               unsigned long long* __restrict__ maxcorr) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g.lox + ci, j = g.loy + blockIdx.y, l = g.loz + blockIdx.z;
    double corr = 0.0;
    if (ci < g.mx) {
        const size_t plane = size_t(g.hx) * g.hy;
        const size_t c = (size_t(l) * g.hy + j) * g.hx + i;
        const double t = T[c];
        double D = 2.0 * (g.ax + g.ay + g.az), radd = 0.0, ff = 1.0;
        // neighbour sums; beyond a convective face the ghost node's T_inner
        // part doubles the inner neighbour (the node is on the face)
        double sx, sy, sz;
        if (i == 0)            { sx = 2.0 * T[c + 1];  D += g.add[0]; radd += g.add[0]; ff *= 2; }
        else if (i == g.hx - 1) { sx = 2.0 * T[c - 1];  D += g.add[1]; radd += g.add[1]; ff *= 2; }
        else                    sx = T[c - 1] + T[c + 1];
        if (j == 0)            { sy = 2.0 * T[c + g.hx]; D += g.add[2]; radd += g.add[2]; ff *= 2; }
        else if (j == g.hy - 1) { sy = 2.0 * T[c - g.hx]; D += g.add[3]; radd += g.add[3]; ff *= 2; }
        else                    sy = T[c - g.hx] + T[c + g.hx];
        if (l == 0)            { sz = 2.0 * T[c + plane]; D += g.add[4]; radd += g.add[4]; ff *= 2; }
        else if (l == g.hz - 1) { sz = 2.0 * T[c - plane]; D += g.add[5]; radd += g.add[5]; ff *= 2; }
        else                    sz = T[c - plane] + T[c + plane];
        // a face node's source density uses its half-size cell (factor 2 per face)
        const double res = g.ax * sx + g.ay * sy + g.az * sz + Q[c] * g.qs * ff +
                           radd * g.tinf - D * t;
        corr = fabs(res / D);
        out[(size_t(blockIdx.z) * g.my + blockIdx.y) * g.mx + ci] = float(res);
    }
    for (int o = 16; o > 0; o >>= 1) corr = fmax(corr, __shfl_xor_sync(0xffffffffu, corr, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(maxcorr, static_cast<unsigned long long>(__double_as_longlong(corr)));
}

// T += e on the unknown nodes.  grid = (ceil(mx / 128), my, mz).
__global__ void k_dir_update(double* __restrict__ T, const float* __restrict__ e, DirGeom g) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= g.mx) return;
    const size_t c = (size_t(g.loz + blockIdx.z) * g.hy + g.loy + blockIdx.y) * g.hx + g.lox + ci;
    T[c] += double(e[(size_t(blockIdx.z) * g.my + blockIdx.y) * g.mx + ci]);
}

// Batched FP32 GEMM C[b] = A[b] B[b] (row-major; batch strides may be 0),
// 64 x 64 output tile per CTA, 16-deep K chunks in shared memory, 4 x 4
// outputs per thread (256 threads).  grid = (ceil(N/64), ceil(M/64), batch).
constexpr int kGemmTile = 64, kGemmK = 16;
__global__ void __launch_bounds__(256) k_dir_gemm(int M, int N, int K, const float* __restrict__ A,
                                                  int lda, size_t sA, const float* __restrict__ B,
                                                  int ldb, size_t sB, float* __restrict__ C,
                                                  int ldc, size_t sC) {
    __shared__ float As[kGemmK][kGemmTile + 4];
    __shared__ float Bs[kGemmK][kGemmTile + 4];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    const int row0 = blockIdx.y * kGemmTile, col0 = blockIdx.x * kGemmTile;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;  // 16 x 16 threads, 4 x 4 each
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kGemmK) {
        // A tile: 64 rows x 16 k (4 per thread), stored k-major
        for (int v = threadIdx.x; v < kGemmTile * kGemmK; v += 256) {
            const int r = v / kGemmK, k = v % kGemmK;
            const int gr = row0 + r, gk = k0 + k;
            As[k][r] = (gr < M && gk < K) ? A[size_t(gr) * lda + gk] : 0.f;
        }
        for (int v = threadIdx.x; v < kGemmTile * kGemmK; v += 256) {
            const int k = v / kGemmTile, c = v % kGemmTile;
            const int gk = k0 + k, gc = col0 + c;
            Bs[k][c] = (gk < K && gc < N) ? B[size_t(gk) * ldb + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kGemmK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][tr + 16 * u];
                b[u] = Bs[k][tc + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = row0 + tr + 16 * u, c = col0 + tc + 16 * v;
            if (r < M && c < N) C[size_t(r) * ldc + c] = acc[u][v];
        }
}

// One tridiagonal solve along z per transverse mode (ky, kx):
//   (2 az + add - lam) e_l - az' e_{l-1} - az'' e_{l+1} = r_l,
// lam = lam_x[kx] + lam_y[ky] (< 0), az' = 2 az in the row of a convective
// end node toward its inner neighbour (Thomas algorithm, FP32, the modified
// super-diagonal kept in `cp`).  In place on w [mz][my][mx].
// grid = ceil(mx my / 128).
__global__ void k_dir_tridiag(float* __restrict__ w, float* __restrict__ cp,
                              const double* __restrict__ lam_x, const double* __restrict__ lam_y,
                              DirGeom g) {
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = g.mx * g.my;
    if (line >= nl) return;
    const int ky = line / g.mx, kx = line - ky * g.mx;
    const float lam = float(lam_x[kx] + lam_y[ky]);
    const float az = float(g.az);
    const int mz = g.mz;
    const bool conv_lo = g.loz == 0, conv_hi = g.loz + mz - 1 == g.hz - 1;
    float cprev = 0.f, dprev = 0.f;
    for (int r = 0; r < mz; ++r) {
        const int l = g.loz + r;
        float b = 2.f * az - lam;
        float a = (r > 0) ? -az : 0.f;          // coefficient of e_{r-1}
        float c = (r < mz - 1) ? -az : 0.f;     // coefficient of e_{r+1}
        if (l == 0 && conv_lo) { b += float(g.add[4]); c = -2.f * az; }
        if (l == g.hz - 1 && conv_hi) { b += float(g.add[5]); a = -2.f * az; }
        const size_t o = size_t(r) * nl + line;
        const float den = b - a * cprev;
        cprev = c / den;
        dprev = (w[o] - a * dprev) / den;
        cp[o] = cprev;
        w[o] = dprev;
    }
    float x = 0.f;
    for (int r = mz - 1; r >= 0; --r) {
        const size_t o = size_t(r) * nl + line;
        x = w[o] - cp[o] * x;
        w[o] = x;
    }
}

// ---------------------------------------------------------------- driver ----

struct HeatDirect {
    DirGeom g;
    float *Vx = nullptr, *VxinvT = nullptr, *VxT = nullptr, *Vy = nullptr, *Vyinv = nullptr;
    double *lam_x = nullptr, *lam_y = nullptr;
    float *w1 = nullptr, *w2 = nullptr, *cp = nullptr;
    unsigned long long* red = nullptr;
};

void free_heat_direct(shg_plan* p) {
    HeatDirect* h = p->hdir;
    if (!h) return;
    void* bufs[] = {h->Vx, h->VxinvT, h->VxT, h->Vy, h->Vyinv, h->lam_x, h->lam_y,
                    h->w1,  h->w2,     h->cp,  h->red};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete h;
    p->hdir = nullptr;
}

static shg_status_t upload_f(float** dst, const std::vector<double>& src) {
    std::vector<float> f(src.begin(), src.end());
    SHG_CK(cudaMalloc((void**)dst, f.size() * sizeof(float)));
    SHG_CK(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    return SHG_OK;
}
static shg_status_t upload_d(double** dst, const std::vector<double>& src) {
    SHG_CK(cudaMalloc((void**)dst, src.size() * sizeof(double)));
    SHG_CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
    return SHG_OK;
}

// (Re)build the eigenbases and work buffers for the plan's heat grid and
// boundary (called when either changes).
shg_status_t heat_direct_setup(shg_plan* p) {
    free_heat_direct(p);
    HeatDirect* h = new HeatDirect();
    p->hdir = h;
    const double kap = p->c.kappa_th;
    const double dx = p->c.wx / (p->g.hx - 1), dy = p->c.wy / (p->g.hy - 1),
                 dz = p->c.L / (p->g.hz - 1);
    const int* f = p->heat_face;
    const double* hh = p->heat_h;
    const Axis X = make_axis(p->g.hx, dx, f[0], f[1], hh[0], hh[1], kap);
    const Axis Y = make_axis(p->g.hy, dy, f[2], f[3], hh[2], hh[3], kap);
    const Axis Z = make_axis(p->g.hz, dz, f[4], f[5], hh[4], hh[5], kap);
    DirGeom& g = h->g;
    g.hx = p->g.hx; g.hy = p->g.hy; g.hz = p->g.hz;
    g.lox = X.lo; g.loy = Y.lo; g.loz = Z.lo;
    g.mx = X.m; g.my = Y.m; g.mz = Z.m;
    g.ax = X.a; g.ay = Y.a; g.az = Z.a;
    g.add[0] = X.add_lo; g.add[1] = X.add_hi; g.add[2] = Y.add_lo; g.add[3] = Y.add_hi;
    g.add[4] = Z.add_lo; g.add[5] = Z.add_hi;
    g.tinf = p->heat_tinf;
    g.qs = 1.0 / (kap * dx * dy * dz);
    std::vector<double> lx, Vx, Vxinv, ly, Vy, Vyinv;
    axis_eigen(X, lx, Vx, Vxinv);
    axis_eigen(Y, ly, Vy, Vyinv);
    const int mx = X.m, my = Y.m;
    std::vector<double> VxinvT(size_t(mx) * mx), VxT(size_t(mx) * mx);
    for (int i = 0; i < mx; ++i)
        for (int k = 0; k < mx; ++k) {
            VxinvT[size_t(i) * mx + k] = Vxinv[size_t(k) * mx + i];
            VxT[size_t(k) * mx + i] = Vx[size_t(i) * mx + k];
        }
    shg_status_t st;
    if ((st = upload_f(&h->VxinvT, VxinvT)) != SHG_OK || (st = upload_f(&h->VxT, VxT)) != SHG_OK ||
        (st = upload_f(&h->Vy, Vy)) != SHG_OK || (st = upload_f(&h->Vyinv, Vyinv)) != SHG_OK ||
        (st = upload_d(&h->lam_x, lx)) != SHG_OK || (st = upload_d(&h->lam_y, ly)) != SHG_OK)
        return st;
    const size_t nw = size_t(g.mx) * g.my * g.mz;
    SHG_CK(cudaMalloc((void**)&h->w1, nw * sizeof(float)));
    SHG_CK(cudaMalloc((void**)&h->w2, nw * sizeof(float)));
    SHG_CK(cudaMalloc((void**)&h->cp, nw * sizeof(float)));
    SHG_CK(cudaMalloc((void**)&h->red, sizeof(unsigned long long)));
    return SHG_OK;
}

static cudaError_t gemm(int M, int N, int K, const float* A, int lda, size_t sA, const float* B,
                        int ldb, size_t sB, float* C, int ldc, size_t sC, int batch,
                        cudaStream_t st) {
    dim3 grid((N + kGemmTile - 1) / kGemmTile, (M + kGemmTile - 1) / kGemmTile, batch);
    k_dir_gemm<<<grid, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
    return cudaGetLastError();
}

// Refine p->theat until the largest Jacobi correction is below tol or
// `max_iters` FP32 solves have been applied.  Returns the final correction
// and the number of solves.
shg_status_t heat_direct_solve(shg_plan* p, int max_iters, double tol, double* resid, int* iters,
                               cudaStream_t st) {
    if (!p->hdir) {
        shg_status_t r = heat_direct_setup(p);
        if (r != SHG_OK) return r;
    }
    HeatDirect* h = p->hdir;
    const DirGeom& g = h->g;
    const int mx = g.mx, my = g.my, mz = g.mz;
    const size_t slab = size_t(mx) * my;
    dim3 pg((mx + 127) / 128, my, mz);
    int n = 0;
    double corr = 0;
    for (;;) {
        SHG_CK(cudaMemsetAsync(h->red, 0, sizeof(unsigned long long), st));
        k_dir_residual<<<pg, 128, 0, st>>>(p->theat, p->Q, g, h->w1, h->red);
        SHG_CK(cudaGetLastError());
        unsigned long long bits = 0;
        SHG_CK(cudaMemcpyAsync(&bits, h->red, sizeof(bits), cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaStreamSynchronize(st));
        memcpy(&corr, &bits, sizeof(double));
        if (!std::isfinite(corr)) return SHG_ERR_NONFINITE;
        if (corr < tol || n >= max_iters) break;
        // r^ = (Vy^-1 (x) Vx^-1) r: along x (all rows of all layers), then along y
        SHG_CK(gemm(my * mz, mx, mx, h->w1, mx, 0, h->VxinvT, mx, 0, h->w2, mx, 0, 1, st));
        SHG_CK(gemm(my, mx, my, h->Vyinv, my, 0, h->w2, mx, slab, h->w1, mx, slab, mz, st));
        k_dir_tridiag<<<(int)((slab + 127) / 128), 128, 0, st>>>(h->w1, h->cp, h->lam_x,
                                                                 h->lam_y, g);
        SHG_CK(cudaGetLastError());
        // e = (Vy (x) Vx) e^
        SHG_CK(gemm(my, mx, my, h->Vy, my, 0, h->w1, mx, slab, h->w2, mx, slab, mz, st));
        SHG_CK(gemm(my * mz, mx, mx, h->w2, mx, 0, h->VxT, mx, 0, h->w1, mx, 0, 1, st));
        k_dir_update<<<pg, 128, 0, st>>>(p->theat, h->w1, g);
        SHG_CK(cudaGetLastError());
        ++n;
    }
    if (resid) *resid = corr;
    if (iters) *iters = n;
    return SHG_OK;
}

}  // namespace shg
