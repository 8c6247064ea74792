// C ABI of libshg: plan management, forward propagation and batched sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "plan.h"

namespace shg {

static thread_local std::string g_last_error;

shg_status_t cuda_fail(cudaError_t e, const char* what) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
    cudaGetLastError();  // clear a non-sticky error so the context stays usable
    return e == cudaErrorMemoryAllocation ? SHG_ERR_OOM : SHG_ERR_CUDA;
}

cudaError_t launch_copy_init(bool fp64, const InitDesc* idescs, int ninst, const void* descs,
                             int nx, int ny, cudaStream_t st);

// Largest per-point temperature table a plan keeps (beyond it the passes
// sample the node table).
constexpr size_t kUmapMaxBytes = size_t(4) << 30;

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

static std::once_flag g_attr_once;
static cudaError_t g_attr_err = cudaSuccess;

static shg_status_t ensure_attributes() {
    std::call_once(g_attr_once, [] { g_attr_err = setup_pass_attributes(); });
    if (g_attr_err != cudaSuccess) return cuda_fail(g_attr_err, "setup_pass_attributes");
    return SHG_OK;
}

// ---------------------------------------------------------- tables ----

static double kvec(int k, int n, double len) {
    // angular frequency of DFT bin k: 2 pi fftfreq(n, len/n)[k]
    const int kk = (k < (n + 1) / 2) ? k : k - n;
    return 2.0 * kPi * kk / len;
}

template <class C> static void put(std::vector<unsigned char>& buf, size_t i, double re, double im) {
    C v;
    v.x = static_cast<decltype(v.x)>(re);
    v.y = static_cast<decltype(v.y)>(im);
    memcpy(buf.data() + i * sizeof(C), &v, sizeof(C));
}

static void put_c(const shg_plan* p, std::vector<unsigned char>& buf, size_t i, double re,
                  double im) {
    if (p->fp64)
        put<double2>(buf, i, re, im);
    else
        put<float2>(buf, i, re, im);
}

// K-space factor entry: double2 in FP64 plans, (hi, lo) float pairs otherwise.
static size_t prop_size(const shg_plan*) { return 16; }  // double2 or float4
static void put_p(const shg_plan* p, std::vector<unsigned char>& buf, size_t i, double re,
                  double im) {
    if (p->fp64) {
        put<double2>(buf, i, re, im);
        return;
    }
    float4 v;
    v.x = float(re);
    v.y = float(im);
    v.z = float(re - double(v.x));
    v.w = float(im - double(v.y));
    memcpy(buf.data() + i * sizeof(float4), &v, sizeof(float4));
}

static shg_status_t upload(void* dst, const std::vector<unsigned char>& src) {
    SHG_CK(cudaMemcpy(dst, src.data(), src.size(), cudaMemcpyHostToDevice));
    return SHG_OK;
}

static double k_f(const shg_plan* p) { return 2 * kPi * p->c.n_f / p->c.lambda_f; }
static double k_sh(const shg_plan* p) { return 2 * kPi * p->c.n_sh / (0.5 * p->c.lambda_f); }

// Row and column K-space factors, with the linear absorption, the walk-off
// phase exp(-i tan(rho_j) Kx dz) (row factor) and the 1/n of the inverse
// transforms folded in (App. A, Eq. (A.4)-(A.5), reading 1).
static shg_status_t build_prop_tables(shg_plan* p) {
    const int nx = p->g.nx, ny = p->g.ny;
    const double dz = p->c.L / p->g.nz;
    const double kj[2] = {k_f(p), k_sh(p)};
    const double al[2] = {p->c.alpha_f, p->c.alpha_sh};
    const double tr[2] = {std::tan(p->c.walkoff_f), std::tan(p->c.walkoff_sh)};  // walk-off
    const size_t ps = prop_size(p);
    std::vector<unsigned char> hx(2 * nx * ps), hy(2 * ny * ps);
    std::vector<unsigned char> hxc(2 * nx * ps), hyc(2 * ny * ps);
    for (int j = 0; j < 2; ++j) {
        const double att = std::exp(-0.5 * al[j] * dz);
        for (int k = 0; k < nx; ++k) {
            const double K = kvec(k, nx, p->g.lx);
            const double ph = -K * K * dz / (2 * kj[j]) - tr[j] * K * dz;
            put_p(p, hx, j * nx + k, att * std::cos(ph) / nx, att * std::sin(ph) / nx);
            put_p(p, hxc, j * nx + k, att * std::cos(ph) / nx, -att * std::sin(ph) / nx);
        }
        for (int k = 0; k < ny; ++k) {
            const double K = kvec(k, ny, p->g.ly);
            const double ph = -K * K * dz / (2 * kj[j]);
            put_p(p, hy, j * ny + k, std::cos(ph) / ny, std::sin(ph) / ny);
            put_p(p, hyc, j * ny + k, std::cos(ph) / ny, -std::sin(ph) / ny);
        }
    }
    shg_status_t st;
    if ((st = upload(p->px, hx)) != SHG_OK) return st;
    if ((st = upload(p->py, hy)) != SHG_OK) return st;
    if ((st = upload(p->pxc, hxc)) != SHG_OK) return st;
    return upload(p->pyc, hyc);
}

DkModel plan_dk_model(const shg_plan* p) {
    DkModel m = p->dkm;
    m.t_ref = m.t_oven + p->b.t_oven_offset;
    return m;
}

// e^{i theta} at every quarter step, theta = (dk0 + g T_off) z, or Dk(T_oven +
// T_off) z with the Eq. (4) model, reduced mod 2 pi.
static shg_status_t build_phase_table(shg_plan* p) {
    const int nq = 4 * p->g.nz + 1;
    const double dq = p->c.L / p->g.nz / 4;
    const DkModel m = plan_dk_model(p);
    const double rate = m.on ? dk_eq4(m, m.t_ref) : p->c.dk0 + p->c.ddk_dT * p->b.t_oven_offset;
    std::vector<unsigned char> h(nq * p->csize);
    for (int q = 0; q < nq; ++q) {
        const double th = std::fmod(rate * (q * dq), 2 * kPi);
        put_c(p, h, q, std::cos(th), std::sin(th));
    }
    return upload(p->eph, h);
}

static shg_status_t build_twiddles(shg_plan* p) {
    std::vector<unsigned char> h(1024 * prop_size(p));
    for (int k = 0; k < 1024; ++k) {
        const double a = -2 * kPi * k / 1024.0;
        put_p(p, h, k, std::cos(a), std::sin(a));
    }
    return upload(p->tw, h);
}

static shg_status_t build_heat_index(shg_plan* p) {
    const int hx = p->g.hx, hy = p->g.hy, hz = p->g.hz;
    const double hdx = p->c.wx / (hx - 1), hdy = p->c.wy / (hy - 1), hdz = p->c.L / (hz - 1);
    std::vector<int> ix(p->g.nx), iy(p->g.ny), lz(p->g.nz + 1);
    for (int m = 0; m < p->g.nx; ++m) {
        const double x = (m - p->g.nx / 2) * (p->g.lx / p->g.nx);
        const int i = int(std::floor((x + p->c.wx / 2) / hdx + 0.5));
        ix[m] = (i >= 0 && i < hx) ? i : -1;
    }
    for (int n = 0; n < p->g.ny; ++n) {
        const double y = (n - p->g.ny / 2) * (p->g.ly / p->g.ny);
        const int j = int(std::floor((y + p->c.wy / 2) / hdy + 0.5));
        iy[n] = (j >= 0 && j < hy) ? j : -1;
    }
    for (int s = 0; s <= p->g.nz; ++s) {
        const double z = s * (p->c.L / p->g.nz);
        const int l = int(std::floor(z / hdz + 0.5));
        lz[s] = (l >= 0 && l < hz) ? l : -1;
    }
    SHG_CK(cudaMemcpy(p->hix, ix.data(), ix.size() * sizeof(int), cudaMemcpyHostToDevice));
    SHG_CK(cudaMemcpy(p->hiy, iy.data(), iy.size() * sizeof(int), cudaMemcpyHostToDevice));
    SHG_CK(cudaMemcpy(p->hlz, lz.data(), lz.size() * sizeof(int), cudaMemcpyHostToDevice));
    return SHG_OK;
}

// ---------------------------------------------------------- tensor maps ----

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// Tensor map of the plan's field buffer seen as 8-byte elements
// [2 fields][ny][nx], with boxes of (column tile) x (up to 256 rows) x 1.
static shg_status_t build_tensor_map(shg_plan* p) {
    const int tile = col_tma_tile(p->fp64, p->g.ny);
    if (tile <= 0) return SHG_OK;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return SHG_OK;  // no driver entry point: the cp.async column pass is used
    const cuuint64_t dims[3] = {cuuint64_t(p->g.nx), cuuint64_t(p->g.ny), 2};
    const cuuint64_t strides[2] = {cuuint64_t(p->g.nx) * 8, cuuint64_t(p->g.nx) * p->g.ny * 8};
    const cuuint32_t box[3] = {cuuint32_t(tile), cuuint32_t(std::min(p->g.ny, 256)), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(&p->cmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, p->field, dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return SHG_OK;  // not encodable: cp.async column pass
    SHG_CK(cudaMalloc(&p->cmap_dev, sizeof(CUtensorMap)));
    SHG_CK(cudaMemcpy(p->cmap_dev, &p->cmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    p->has_cmap = true;
    return SHG_OK;
}

// ------------------------------------------------------ descriptors ----

template <class R> static void fill_desc(const shg_plan* p, InstDesc<R>* d, void* field) {
    memset(d, 0, sizeof(*d));
    const double lam_f = p->c.lambda_f, lam_s = 0.5 * p->c.lambda_f;
    const double cF = 0.5 * kEps0 * kCLight * p->c.n_f;
    const double cS = 0.5 * kEps0 * kCLight * p->c.n_sh;
    d->field = static_cast<cx<R>*>(field);
    d->px = static_cast<const pt<R>*>(p->px);
    d->py = static_cast<const pt<R>*>(p->py);
    d->eph = static_cast<const cx<R>*>(p->eph);
    d->ttab = static_cast<const cx<R>*>(p->ttab);
    d->umap = (!p->fp64 && p->ttab) ? static_cast<const cx<R>*>(p->umap) : nullptr;
    d->tx = p->tx;
    d->ty = p->ty;
    d->tz = p->tz;
    if (p->ttab) {
        d->tx0 = R(-p->tlx / 2);
        d->ty0 = R(-p->tly / 2);
        d->tdx_inv = R((p->tx - 1) / p->tlx);
        d->tdy_inv = R((p->ty - 1) / p->tly);
        d->tdz_inv = R((p->tz - 1) / p->c.L);
    }
    d->dx = R(p->g.lx / p->g.nx);
    d->dy = R(p->g.ly / p->g.ny);
    d->x0 = R(-(p->g.nx / 2) * (p->g.lx / p->g.nx));
    d->y0 = R(-(p->g.ny / 2) * (p->g.ly / p->g.ny));
    d->kF = R(2 * kPi * p->c.d_eff / (p->c.n_f * lam_f));
    d->kS = R(2 * kPi * p->c.d_eff / (p->c.n_sh * lam_f));
    d->bF = R(0.5 * p->c.beta_f * cF);
    d->bS = R(0.5 * p->c.beta_sh * cS);
    d->lF = R(2 * kPi / lam_f * p->c.dn_dT);
    d->lS = R(2 * kPi / lam_s * p->c.dn_dT);
    d->psi0F = R(2 * kPi / lam_f * p->c.dn_dT * p->b.t_oven_offset);
    d->psi0S = R(2 * kPi / lam_s * p->c.dn_dT * p->b.t_oven_offset);
    // the phase is theta(z) + g C: with the Eq. (4) model the table's C already
    // holds the integral of Dk (g = 1); without a map g is the slope dDk/dT at
    // T_oven + T_off, which only the adjoint's oven-offset gradient uses
    if (p->dkm.on) {
        const DkModel m = plan_dk_model(p);
        d->g = R(p->ttab ? 1.0 : dk_eq4_slope(m, m.t_ref));
    } else {
        d->g = R(p->c.ddk_dT);
    }
    d->dz = R(p->c.L / p->g.nz);
    d->undepleted = p->b.undepleted ? 1 : 0;
    d->status = p->status;
    d->wait_polls = p->wait_polls;
    d->mon = p->mon;
    d->mon_every = p->mon_every > 0 ? p->mon_every : 1;
    d->mon_last = p->mon_slots - 1;
    if ((p->flags & SHG_FLAG_THERMAL) && p->Q) {
        d->Q = p->Q;
        d->hix = p->hix;
        d->hiy = p->hiy;
        d->hlz = p->hlz;
        d->hx = p->g.hx;
        d->hy = p->g.hy;
        d->hz = p->g.hz;
        d->qaF = R(p->c.alpha_f * cF);
        d->qbF = R(p->c.beta_f * cF * cF);
        d->qaS = R(p->c.alpha_sh * cS);
        d->qbS = R(p->c.beta_sh * cS * cS);
        d->dxdy = R((p->g.lx / p->g.nx) * (p->g.ly / p->g.ny));
    }
}

void fill_desc_f32(const shg_plan* p, InstDesc<float>* d) { fill_desc<float>(p, d, p->field); }
void fill_desc_f64(const shg_plan* p, InstDesc<double>* d) { fill_desc<double>(p, d, p->field); }

void fill_init(const shg_plan* p, InitDesc* d) {
    memset(d, 0, sizeof(*d));
    d->dx = p->g.lx / p->g.nx;
    d->dy = p->g.ly / p->g.ny;
    d->x0 = -(p->g.nx / 2) * d->dx;
    d->y0 = -(p->g.ny / 2) * d->dy;
    d->w0 = p->b.w0;
    d->zf = p->b.z_focus;
    d->kF = k_f(p);
    d->p1 = p->b.p1;
    d->cFdxdy = 0.5 * kEps0 * kCLight * p->c.n_f * d->dx * d->dy;
    d->cSdxdy = 0.5 * kEps0 * kCLight * p->c.n_sh * d->dx * d->dy;
    d->red = p->red;
    d->pw = p->pw;
    d->f0 = p->custom_init ? p->field0 : nullptr;
}

static size_t desc_bytes(bool fp64) { return fp64 ? sizeof(InstDesc<double>) : sizeof(InstDesc<float>); }

static void fill_desc_any(const shg_plan* p, void* out) {
    if (p->fp64)
        fill_desc_f64(p, static_cast<InstDesc<double>*>(out));
    else
        fill_desc_f32(p, static_cast<InstDesc<float>*>(out));
}

static shg_status_t upload_desc(shg_plan* p) {
    std::vector<unsigned char> h(desc_bytes(p->fp64));
    fill_desc_any(p, h.data());
    SHG_CK(cudaMemcpy(p->desc, h.data(), h.size(), cudaMemcpyHostToDevice));
    InitDesc id;
    fill_init(p, &id);
    SHG_CK(cudaMemcpy(p->idesc, &id, sizeof(id), cudaMemcpyHostToDevice));
    if (p->w3) return upload_desc3(p);
    return SHG_OK;
}

// Wait (host) for the plan's last propagation and for a table rebuild still
// in flight, before a call rewrites state that device work may be reading.
static shg_status_t quiesce(shg_plan* p) {
    if (p->last_stream != nullptr || p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    if (p->ready_pending) {
        SHG_CK(cudaEventSynchronize(p->ready));
        p->ready_pending = false;
    }
    return SHG_OK;
}

// ----------------------------------------------------------- forward ----

// ---------------------------------------------------------- autotuner ----

static std::mutex g_tune_mu;
static std::map<std::tuple<bool, int, int>, int> g_tuned;
static bool g_cache_loaded = false;

// Optional persistent tuner decisions: with SHG_TUNE_CACHE=<file>, decisions
// found in the file are used instead of timing, and new decisions are
// appended ("fp64 n key flavour" per line; key as tune_key: 0 row, 1 column,
// 2 row with the per-point table, +4 for groups of few instances).  Caller
// holds g_tune_mu.
static void load_tune_cache() {
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char* path = getenv("SHG_TUNE_CACHE");
    if (!path || !path[0]) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    int fp64, n, pass, v;
    while (fscanf(f, "%d %d %d %d", &fp64, &n, &pass, &v) == 4)
        if (v >= 0 && v <= 5) g_tuned.emplace(std::make_tuple(fp64 != 0, n, pass), v);  // flavours 0-5
    fclose(f);
}
static void save_tune_decision(bool fp64, int n, int pass, int v) {
    const char* path = getenv("SHG_TUNE_CACHE");
    if (!path || !path[0]) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d\n", fp64 ? 1 : 0, n, pass, v);
    fclose(f);
}

static int forced_variant() {
    const char* f = getenv("SHG_FFT_VARIANT");
    return (f && f[0] >= '0' && f[0] <= '5' && f[1] == 0) ? f[0] - '0' : -1;
}

static bool p_fp32(const std::vector<shg_plan*>& plans) {
    for (const shg_plan* p : plans)
        if (p->fp64) return false;
    return true;
}

int row_umap_bit(const std::vector<shg_plan*>& plans) {
    bool any = false, extras = false;
    for (const shg_plan* p : plans) {
        extras |= p->mon != nullptr;
        if (!p->ttab) continue;
        if (!p->umap || !(double(p->tz - 1) < 0.99 * p->g.nz)) return 0;
        any = true;
    }
    if (!any) return 0;
    const char* v = getenv("SHG_ROW_LEAN");  // 0: always the instantiation with the z_s code
    const bool lean_ok = !(v && v[0] == '0');
    return (lean_ok && p_fp32(plans) && !extras) ? (kRowUmap | kRowLean) : kRowUmap;
}

// The one-pass-per-step schedule (k_col_step): FP32 groups on the per-point
// table without monitors (the monitor-free rows) or adjoint checkpoints (the
// adjoint replays the two-pass states).  Heat deposits are binned in either
// layout.  SHG_STEP_PASSES=0 keeps two passes per step.
static bool step_schedule(bool fp64, const std::vector<shg_plan*>& plans, int rb) {
    const char* v = getenv("SHG_STEP_PASSES");
    if (v && v[0] == '0') return false;
    if (fp64 || (rb & (kRowUmap | kRowLean)) != (kRowUmap | kRowLean)) return false;
    for (const shg_plan* p : plans)
        if (p->adj) return false;
    return true;
}

static_assert(kRowUmap > 5 && kRowLean > 5 && kRowLean != kRowUmap,
              "the row-pass bits must not collide with a flavour number");

// Candidate flavours of a pass for a length: the default shape, the
// alternative shape, the default shape in 128-thread CTAs and (column pass)
// the TMA-staged kernel and the default shape in 512-thread CTAs.
static std::vector<int> candidates(bool fp64, int n, int pass, bool tmaps) {
    std::vector<int> c{0};
    if (has_fft_variant(fp64, n)) c.push_back(1);
    if (pass == 1 && tmaps && col_tma_tile(fp64, n) > 0) c.push_back(2);
    // flavour 4 (64-thread CTAs) is not a candidate: its launches time well
    // alone, but whole single-instance propagations (graph, programmatic
    // launches) measured slower with it; SHG_FFT_VARIANT=4 still selects it
    if (has_col_small(fp64, n)) c.push_back(3);
    if (pass == 1 && has_col_wide(fp64, n)) c.push_back(5);
    return c;
}

// Tuner key of a pass: 0 row, 1 column, 2 row with the per-point table; +4
// for groups of at most kFewInstances instances (decided separately, since
// small CTAs pay off there and not in large batches).
constexpr int kFewInstances = 8;
static int tune_key(int pass, int row_bits, int ninst) {
    return pass + (pass == 0 && row_bits ? 2 : 0) + (ninst <= kFewInstances ? 4 : 0);
}

// A flavour this (precision, length, pass) does not have becomes flavour 0
// (a forced flavour, or a decision read from a tuner cache of another build).
static int supported_flavour(bool fp64, int n, int pass, int f) {
    if (f == 1 && !has_fft_variant(fp64, n)) return 0;
    if (f == 2 && pass == 0) return 0;
    if (f == 5) return (pass == 1 && has_col_wide(fp64, n)) ? 5 : 0;
    if (f >= 3 && !has_col_small(fp64, n)) return 0;
    return f;
}

// Tuner keys of the one-pass-per-step kernels: 8 the row-layout pass, 9 the
// column-layout pass (+4 for groups of at most kFewInstances instances).
static int step_key(int which, int ninst) { return 8 + which + (ninst <= kFewInstances ? 4 : 0); }

// Flavour of a step kernel: which = 0, the row-layout pass (row flavours 0,
// 1, 3, 4); which = 1, the column-layout pass (1: the 8-element shape, 3:
// 128-thread CTAs, 5: 512-thread CTAs, where they exist, else 0).
static int supported_step_flavour(bool fp64, int n, int which, int f) {
    if (which == 0) return supported_flavour(fp64, n, 0, f == 2 || f == 5 ? 0 : f);
    if (f == 5) return has_col_step_wide(n) ? 5 : 0;
    if (f == 1) return has_col_step_v1(n) ? 1 : 0;
    return (f == 3 || f == 4) && has_col_step_small(n) ? 3 : 0;
}

int step_variant(bool fp64, int n, int which, int ninst) {
    const int f = forced_variant();
    if (f >= 0) return supported_step_flavour(fp64, n, which, f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_cache();
    auto it = g_tuned.find(std::make_tuple(fp64, n, step_key(which, ninst)));
    return it == g_tuned.end() ? 0 : supported_step_flavour(fp64, n, which, it->second);
}

int fft_variant(bool fp64, int n, int pass, int row_bits, int ninst) {
    const int f = forced_variant();
    if (f >= 0) return supported_flavour(fp64, n, pass, f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_cache();
    auto it = g_tuned.find(std::make_tuple(fp64, n, tune_key(pass, row_bits, ninst)));
    return it == g_tuned.end() ? 0 : supported_flavour(fp64, n, pass, it->second);
}

// The tuner's two timing events, released on every return.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Time every candidate flavour of each pass of this group on its own data and
// keep the fastest for the rest of the process.  After one warm-up launch
// each, the candidates take turns for three rounds of two launches (CUDA
// events on `st`), so that none profits from caches the others warmed; a
// candidate's time is its best round.  The group's fields are modified; every
// propagation re-initialises them first.
shg_status_t tune_group(bool fp64, int nx, int ny, int nz, const void* descs, int ninst,
                        const void* tw, int hx, cudaStream_t st, const void* tmaps, int row_bits,
                        bool steps, int hy) {
    if (forced_variant() >= 0) return SHG_OK;
    steps = steps && nz >= 3;  // the step kernels are timed at s = 2 (rows) and s = 1 (columns)
    // passes: 0 rows, 1 the column pass of the two-pass schedule; with one
    // pass per step, 0 the row-layout and 2 the column-layout step pass
    for (int pass = 0; pass < 3; ++pass) {
        if ((pass == 1 && steps) || (pass == 2 && !steps)) continue;
        const int n = pass == 0 ? nx : ny;
        std::vector<int> cand;
        if (pass == 2) {
            cand.push_back(0);
            if (has_col_step_v1(n)) cand.push_back(1);
            if (has_col_step_small(n)) cand.push_back(3);
            if (has_col_step_wide(n)) cand.push_back(5);
        } else {
            cand = candidates(fp64, n, pass, tmaps != nullptr && !steps);
        }
        if (cand.size() < 2) continue;
        const int key = steps ? step_key(pass == 0 ? 0 : 1, ninst) : tune_key(pass, row_bits, ninst);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            load_tune_cache();
            if (g_tuned.count(std::make_tuple(fp64, n, key))) continue;
        }
        EventPair ev;
        SHG_CK(cudaEventCreate(&ev.e0));
        SHG_CK(cudaEventCreate(&ev.e1));
        cudaEvent_t e0 = ev.e0, e1 = ev.e1;
        const int s = nz > 1 ? 1 : 0;
        auto launch = [&](int v) {
            if (steps)
                return pass == 0 ? launch_row_step(nx, descs, ninst, ny, nz, 2, tw, hx, st, v | row_bits)
                                 : launch_col_step(ny, descs, ninst, nx, nz, 1, tw, hy, st, v);
            return pass == 0 ? launch_row(fp64, nx, descs, ninst, ny, nz, s, tw, hx, st, v | row_bits)
                             : launch_col(fp64, ny, descs, ninst, nx, tw, st, v, tmaps);
        };
        std::vector<float> best(cand.size(), 1e30f);
        for (int v : cand) {
            const cudaError_t e = launch(v);
            if (e != cudaSuccess) return cuda_fail(e, "tune_group");
        }
        for (int round = 0; round < 3; ++round) {
            for (size_t c = 0; c < cand.size(); ++c) {
                SHG_CK(cudaEventRecord(e0, st));
                for (int rep = 0; rep < 2; ++rep) {
                    const cudaError_t e = launch(cand[c]);
                    if (e != cudaSuccess) return cuda_fail(e, "tune_group");
                }
                SHG_CK(cudaEventRecord(e1, st));
                SHG_CK(cudaEventSynchronize(e1));
                float t = 0;
                SHG_CK(cudaEventElapsedTime(&t, e0, e1));
                best[c] = std::min(best[c], t);
            }
        }
        int best_v = cand[0];
        float best_t = best[0];
        for (size_t c = 1; c < cand.size(); ++c)
            if (best[c] < best_t) {
                best_t = best[c];
                best_v = cand[c];
            }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_tuple(fp64, n, key)] = best_v;
        save_tune_decision(fp64, n, key, best_v);
    }
    return SHG_OK;
}

shg_status_t enqueue_forward(bool fp64, int nx, int ny, int nz, const void* descs,
                             const InitDesc* idescs, int ninst, const void* tw,
                             const std::vector<shg_plan*>& plans, cudaStream_t st,
                             const void* tmaps, int* status_arr) {
    const bool custom = plans[0]->custom_init;
    if (status_arr) {
        const cudaError_t e0 = cudaMemsetAsync(status_arr, 0, ninst * sizeof(int), st);
        if (e0 != cudaSuccess) return cuda_fail(e0, "memset status");
    } else {
        for (shg_plan* p : plans) {
            const cudaError_t e0 = cudaMemsetAsync(p->status, 0, sizeof(int), st);
            if (e0 != cudaSuccess) return cuda_fail(e0, "memset status");
        }
    }
    for (shg_plan* p : plans) {
        if (p->mon) {
            const cudaError_t e0 = cudaMemsetAsync(p->mon, 0, 2 * p->mon_slots * sizeof(double), st);
            if (e0 != cudaSuccess) return cuda_fail(e0, "memset monitor");
        }
    }
    cudaError_t e = custom ? launch_copy_init(fp64, idescs, ninst, descs, nx, ny, st)
                           : launch_init(fp64, idescs, nullptr, ninst, descs, nx, ny, st);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    for (shg_plan* p : plans) {
        if ((p->flags & SHG_FLAG_THERMAL) && p->Q) {
            e = cudaMemsetAsync(p->Q, 0, sizeof(double) * p->g.hx * p->g.hy * p->g.hz, st);
            if (e != cudaSuccess) return cuda_fail(e, "memset Q");
        }
    }
    int hx = 0, hy = 0;
    for (shg_plan* p : plans)
        if ((p->flags & SHG_FLAG_THERMAL) && p->Q) {
            hx = std::max(hx, p->g.hx);
            hy = std::max(hy, p->g.hy);
        }
    if (cluster_path(plans)) {
        // the whole z-march in one cluster-resident launch
        e = launch_cluster(nx, descs, ninst, nz, tw, st);
        if (e != cudaSuccess) return cuda_fail(e, "cluster propagation");
        e = launch_power(fp64, idescs, descs, ninst, nx, ny, st);
        if (e != cudaSuccess) return cuda_fail(e, "power");
        return SHG_OK;
    }
    const int rb = row_umap_bit(plans);
    const int vr = fft_variant(fp64, nx, 0, rb, ninst) | rb;
    const int vc = fft_variant(fp64, ny, 1, 0, ninst);
    if (step_schedule(fp64, plans, rb)) {
        // one pass per step: rows (even s) and columns (odd s) alternate
        const int vrs = step_variant(fp64, nx, 0, ninst) | rb;
        const int vcs = step_variant(fp64, ny, 1, ninst);
        for (int s = 0; s <= nz; ++s) {
            if (s == 0)
                e = launch_row(fp64, nx, descs, ninst, ny, nz, 0, tw, hx, st, vrs);
            else if ((s & 1) == 0)
                e = launch_row_step(nx, descs, ninst, ny, nz, s, tw, hx, st, vrs);
            else
                e = launch_col_step(ny, descs, ninst, nx, nz, s, tw, hy, st, vcs);
            if (e != cudaSuccess) return cuda_fail(e, "step pass");
        }
        e = launch_power(fp64, idescs, descs, ninst, nx, ny, st);
        if (e != cudaSuccess) return cuda_fail(e, "power");
        return SHG_OK;
    }
    for (int s = 0; s <= nz; ++s) {
        for (shg_plan* p : plans) {
            shg_status_t r = adjoint_checkpoint(p, s, st);
            if (r != SHG_OK) return r;
        }
        e = launch_row(fp64, nx, descs, ninst, ny, nz, s, tw, hx, st, vr);
        if (e != cudaSuccess) return cuda_fail(e, "row pass");
        if (s < nz) {
            e = launch_col(fp64, ny, descs, ninst, nx, tw, st, vc, tmaps);
            if (e != cudaSuccess) return cuda_fail(e, "column pass");
        }
    }
    e = launch_power(fp64, idescs, descs, ninst, nx, ny, st);
    if (e != cudaSuccess) return cuda_fail(e, "power");
    return SHG_OK;
}

static bool use_graphs() {
    const char* v = getenv("SHG_NO_GRAPH");
    return !(v && v[0] == '1');
}

// Capture `fn(stream)` into an executable graph using the private stream.
template <class Fn>
static shg_status_t capture(cudaStream_t cap, Fn fn, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    SHG_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    shg_status_t st = fn(cap);
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (st != SHG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    // node priorities: the pass launches of a batch's largest group carry one
    e = cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return SHG_OK;
}

static shg_status_t plan_forward(shg_plan* p, cudaStream_t st) {
    if (p->w3) {
        // three-wave mixing: its own passes, captured into the plan's graph,
        // with programmatic dependent launch between them
        PdlScope pdl(true);
        auto body3 = [&](cudaStream_t q) { return enqueue_forward3(p, q); };
        if (!use_graphs()) return body3(st);
        if (!p->gvalid) {
            if (p->gexec) {
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
            shg_status_t r = capture(p->cap, body3, &p->gexec);
            if (r != SHG_OK) return r;
            p->gvalid = true;
        }
        SHG_CK(cudaGraphLaunch(p->gexec, st));
        return SHG_OK;
    }
    std::vector<shg_plan*> one{p};
    PdlScope pdl(true);  // one grid group
    const void* tmaps = p->has_cmap ? p->cmap_dev : nullptr;
    auto body = [&](cudaStream_t s) {
        return enqueue_forward(p->fp64, p->g.nx, p->g.ny, p->g.nz, p->desc, p->idesc, 1, p->tw,
                               one, s, tmaps);
    };
    if (!cluster_path(one)) {
        const bool dep = (p->flags & SHG_FLAG_THERMAL) && p->Q;
        const int rb = row_umap_bit(one);
        shg_status_t r = tune_group(p->fp64, p->g.nx, p->g.ny, p->g.nz, p->desc, 1, p->tw,
                                    dep ? p->g.hx : 0, st, p->has_cmap ? p->cmap_dev : nullptr, rb,
                                    step_schedule(p->fp64, one, rb), dep ? p->g.hy : 0);
        if (r != SHG_OK) return r;
    }
    if (!use_graphs()) return body(st);
    if (!p->gvalid) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        shg_status_t s = capture(p->cap, body, &p->gexec);
        if (s != SHG_OK) return s;
        p->gvalid = true;
    }
    SHG_CK(cudaGraphLaunch(p->gexec, st));
    return SHG_OK;
}

}  // namespace shg

using namespace shg;

// ============================================================ C ABI ====

extern "C" {

const char* shg_status_string(shg_status_t s) {
    switch (s) {
        case SHG_OK: return "ok";
        case SHG_ERR_INVALID_ARG: return "invalid argument";
        case SHG_ERR_UNSUPPORTED_GRID: return "unsupported grid (nx, ny must be powers of two in [8, 1024]; [8, 256] in FP64)";
        case SHG_ERR_OOM: return "device allocation failed";
        case SHG_ERR_CUDA: return "CUDA error";
        case SHG_ERR_TIMEOUT: return "device-side wait timed out";
        case SHG_ERR_NONFINITE: return "non-finite power or efficiency";
        case SHG_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* shg_last_error(void) { return g_last_error.c_str(); }

static void plan_free(shg_plan* p);

// The map tables of an Eq. (4) plan depend on T_oven + T_off: rebuild them
// (synchronously) after a change of either.
static shg_status_t rebuild_model_tables(shg_plan* p) {
    if (!p->dkm.on || !p->ttab) return SHG_OK;
    SHG_CK(launch_build_ttab(p->fp64, p->tmap, p->ttab, p->tx, p->ty, p->tz,
                             p->c.L / (p->tz - 1), plan_dk_model(p), nullptr));
    if (p->umap) SHG_CK(launch_upsample_map(p->desc, p->umap, p->g.nx, p->g.ny, p->tz, nullptr));
    SHG_CK(cudaStreamSynchronize(nullptr));
    return SHG_OK;
}

// Non-null and pairwise distinct: the same plan twice in one call would have
// two instances write its fields (or rebuild its tables) at once.
static bool distinct_plans(shg_plan* const* plans, int n) {
    std::vector<shg_plan*> v(plans, plans + n);
    std::sort(v.begin(), v.end());
    if (!v.empty() && v.front() == nullptr) return false;
    return std::adjacent_find(v.begin(), v.end()) == v.end();
}

// Largest nz: the stage index 4 s + q of the kernels stays far inside int.
constexpr int kMaxNz = 1 << 26;

static bool finite_beams(const shg_beams_t* b) {
    return std::isfinite(b->p1) && std::isfinite(b->w0) && std::isfinite(b->z_focus) &&
           std::isfinite(b->t_oven_offset) && b->w0 > 0 && b->p1 >= 0;
}

static bool finite_crystal(const shg_crystal_t* c) {
    const double v[] = {c->L,      c->lambda_f, c->n_f,      c->n_sh,       c->d_eff,
                        c->alpha_f, c->alpha_sh, c->beta_f,  c->beta_sh,    c->dk0,
                        c->ddk_dT, c->dn_dT,    c->kappa_th, c->wx,         c->wy,
                        c->walkoff_f, c->walkoff_sh};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

shg_status_t shg_plan_create(const shg_grid_t* grid, const shg_crystal_t* crystal,
                             const shg_beams_t* beams, int flags, shg_plan_t** out) {
    if (out) *out = nullptr;
    if (!grid || !crystal || !beams || !out) return SHG_ERR_INVALID_ARG;
    const bool fp64 = (flags & SHG_FLAG_FP64) != 0;
    const int hi = fp64 ? 256 : 1024;
    if (!pow2_in(grid->nx, 8, hi) || !pow2_in(grid->ny, 8, hi)) return SHG_ERR_UNSUPPORTED_GRID;
    if (grid->nz < 1 || grid->nz > kMaxNz || !(grid->lx > 0) || !(grid->ly > 0) ||
        !std::isfinite(grid->lx) || !std::isfinite(grid->ly))
        return SHG_ERR_INVALID_ARG;
    if (!finite_crystal(crystal) || !finite_beams(beams)) return SHG_ERR_INVALID_ARG;
    if (!(crystal->L > 0) || !(crystal->lambda_f > 0) || !(crystal->n_f > 0) ||
        !(crystal->n_sh > 0) ||
        !(std::fabs(crystal->walkoff_f) < 1.5) || !(std::fabs(crystal->walkoff_sh) < 1.5))
        return SHG_ERR_INVALID_ARG;
    if (flags & SHG_FLAG_THERMAL) {
        if (grid->hx < 3 || grid->hy < 3 || grid->hz < 3 || !(crystal->wx > 0) ||
            !(crystal->wy > 0) || !(crystal->kappa_th > 0))
            return SHG_ERR_INVALID_ARG;
        // the row pass bins the heat deposit per CTA in shared memory
        for (int v : {0, 1, 3, 4, kRowUmap, 1 | kRowUmap, 3 | kRowUmap, 4 | kRowUmap})
            if (row_pass_smem(fp64, grid->nx, grid->hx, v) > 223 * 1024)
                return SHG_ERR_UNSUPPORTED_GRID;
    }
    shg_status_t st = ensure_attributes();
    if (st != SHG_OK) return st;
    shg_plan* p = new shg_plan();
    p->g = *grid;
    p->c = *crystal;
    p->b = *beams;
    p->flags = flags;
    p->fp64 = fp64;
    p->csize = fp64 ? 16 : 8;
    cudaGetDevice(&p->device);
    const size_t npts = size_t(grid->nx) * grid->ny;
    auto fail = [&](cudaError_t e, const char* what) {
        shg_status_t s = cuda_fail(e, what);
        plan_free(p);
        return s;
    };
    cudaError_t e;
#define ALLOC(ptr, bytes)                                                   \
    if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) return fail(e, "cudaMalloc " #ptr);
    ALLOC(p->field, 2 * npts * p->csize);
    ALLOC(p->px, 2 * grid->nx * 16);
    ALLOC(p->py, 2 * grid->ny * 16);
    ALLOC(p->pxc, 2 * grid->nx * 16);
    ALLOC(p->pyc, 2 * grid->ny * 16);
    ALLOC(p->eph, (4 * size_t(grid->nz) + 1) * p->csize);
    ALLOC(p->tw, 1024 * 16);
    ALLOC(p->desc, desc_bytes(fp64));
    ALLOC(p->idesc, sizeof(InitDesc));
    ALLOC(p->red, 2 * kRedBlocks * sizeof(double));
    ALLOC(p->pw, 2 * sizeof(double));
    ALLOC(p->status, sizeof(int));
    if ((e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e, "cudaEventCreate");
    if (flags & SHG_FLAG_THERMAL) {
        const size_t nh = size_t(grid->hx) * grid->hy * grid->hz;
        ALLOC(p->Q, nh * sizeof(double));
        ALLOC(p->theat, nh * sizeof(double));
        ALLOC(p->theat_prev, nh * sizeof(double));
        ALLOC(p->theat_f, nh * sizeof(float));
        ALLOC(p->hix, grid->nx * sizeof(int));
        ALLOC(p->hiy, grid->ny * sizeof(int));
        ALLOC(p->hlz, (grid->nz + 1) * sizeof(int));
        ALLOC(p->hred, 2 * 1024 * sizeof(double));
        if ((e = cudaMemset(p->Q, 0, nh * sizeof(double))) != cudaSuccess) return fail(e, "memset");
        if ((e = cudaMemset(p->theat, 0, nh * sizeof(double))) != cudaSuccess) return fail(e, "memset");
        if ((e = cudaMemset(p->theat_prev, 0, nh * sizeof(double))) != cudaSuccess)
            return fail(e, "memset");
    }
#undef ALLOC
    if ((e = cudaMemset(p->field, 0, 2 * npts * p->csize)) != cudaSuccess) return fail(e, "memset");
    if ((e = cudaMemset(p->status, 0, sizeof(int))) != cudaSuccess) return fail(e, "memset");
    if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(e, "cudaStreamCreate");
    if ((st = build_prop_tables(p)) != SHG_OK || (st = build_phase_table(p)) != SHG_OK ||
        (st = build_tensor_map(p)) != SHG_OK ||
        (st = build_twiddles(p)) != SHG_OK ||
        ((flags & SHG_FLAG_THERMAL) && (st = build_heat_index(p)) != SHG_OK) ||
        // eigenbases of the direct heat solve for the default (oven-held) faces
        ((flags & SHG_FLAG_THERMAL) && (st = heat_direct_setup(p)) != SHG_OK) ||
        (st = upload_desc(p)) != SHG_OK ||
        ((flags & SHG_FLAG_ADJOINT) && (st = adjoint_alloc(p)) != SHG_OK)) {
        plan_free(p);
        return st;
    }
    *out = p;
    return SHG_OK;
}


static void plan_free(shg_plan* p) {
    if (!p) return;
    shg::forget_plan_batches(p);
    shg::free_adjoint(p);
    shg::free_heat_direct(p);
    shg::free_three_wave(p);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->done) cudaEventDestroy(p->done);
    if (p->ready) cudaEventDestroy(p->ready);
    void* bufs[] = {p->field, p->field0, p->px,  p->py,  p->pxc,  p->pyc,   p->eph,
                    p->tw,    p->ttab,   p->umap, p->tmap, p->desc, p->idesc, p->red, p->pw,
                    p->Q,     p->hix,    p->hiy, p->hlz,  p->theat, p->theat_prev, p->theat_f,
                    p->hred,  p->status, p->cmap_dev, p->mon};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete p;
}

shg_status_t shg_plan_destroy(shg_plan_t* p) {
    if (!p) return SHG_OK;
    if (p->has_result || p->last_stream) cudaStreamSynchronize(p->last_stream);
    if (p->ready_pending) cudaEventSynchronize(p->ready);  // a table rebuild in flight
    plan_free(p);
    return SHG_OK;
}

shg_status_t shg_set_wait_limit(shg_plan_t* p, unsigned polls) {
    if (!p) return SHG_ERR_INVALID_ARG;
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    p->wait_polls = polls;
    return upload_desc(p);
}

shg_status_t shg_set_beams(shg_plan_t* p, const shg_beams_t* beams) {
    if (!p || !beams || !finite_beams(beams) || p->w3) return SHG_ERR_INVALID_ARG;
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    adjoint_forward_state(p, false);
    p->b = *beams;
    if (p->custom_init) {
        p->custom_init = false;
        p->gvalid = false;
    }
    if ((st = build_phase_table(p)) != SHG_OK) return st;
    if ((st = upload_desc(p)) != SHG_OK) return st;
    return rebuild_model_tables(p);
}

shg_status_t shg_set_temperature(shg_plan_t* p, const float* dT_dev, int tx, int ty, int tz,
                                 double t_lx, double t_ly, shg_stream_t stream) {
    if (!p) return SHG_ERR_INVALID_ARG;
    // every argument is checked before anything of the plan changes: a refused
    // call leaves the map, the tables and the adjoint checkpoints as they were
    if (dT_dev != nullptr &&
        (tx < 2 || ty < 2 || tz < 2 || !std::isfinite(t_lx) || !std::isfinite(t_ly)))
        return SHG_ERR_INVALID_ARG;
    adjoint_forward_state(p, false);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Fast path: a new map of the shape and extent already installed.  The
    // tables are rebuilt in place, stream-ordered after the last propagation
    // (event), with no host synchronisation and no descriptor change.
    if (dT_dev != nullptr && p->ttab != nullptr && p->tx == tx && p->ty == ty && p->tz == tz &&
        p->tlx == (t_lx > 0 ? t_lx : p->g.lx) && p->tly == (t_ly > 0 ? t_ly : p->g.ly)) {
        const size_t n = size_t(tx) * ty * tz;
        if (p->done_valid) SHG_CK(cudaStreamWaitEvent(s, p->done, 0));
        // after a rebuild still in flight on another stream (same tables)
        if (p->ready_pending) SHG_CK(cudaStreamWaitEvent(s, p->ready, 0));
        if (dT_dev != p->tmap)
            SHG_CK(cudaMemcpyAsync(p->tmap, dT_dev, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                   s));
        SHG_CK(launch_build_ttab(p->fp64, p->tmap, p->ttab, tx, ty, tz, p->c.L / (tz - 1),
                                 plan_dk_model(p), s));
        if (p->umap) SHG_CK(launch_upsample_map(p->desc, p->umap, p->g.nx, p->g.ny, tz, s));
        SHG_CK(cudaEventRecord(p->ready, s));
        p->ready_pending = true;
        return SHG_OK;
    }
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    if (p->ready_pending) {
        SHG_CK(cudaEventSynchronize(p->ready));
        p->ready_pending = false;
    }
    if (dT_dev == nullptr) {
        if (p->ttab) {
            cudaFree(p->ttab);
            cudaFree(p->tmap);
            p->ttab = nullptr;
            p->tmap = nullptr;
            p->tx = p->ty = p->tz = 0;
            p->gvalid = false;
        }
        if (p->umap) {
            cudaFree(p->umap);
            p->umap = nullptr;
            p->umap_bytes = 0;
        }
        return upload_desc(p);
    }
    const size_t n = size_t(tx) * ty * tz;
    if (p->ttab == nullptr || p->tx != tx || p->ty != ty || p->tz != tz) {
        if (p->ttab) cudaFree(p->ttab);
        if (p->tmap) cudaFree(p->tmap);
        p->ttab = nullptr;
        p->tmap = nullptr;
        SHG_CK(cudaMalloc((void**)&p->ttab, n * p->csize));
        SHG_CK(cudaMalloc((void**)&p->tmap, n * sizeof(float)));
        p->gvalid = false;
    }
    p->tx = tx;
    p->ty = ty;
    p->tz = tz;
    p->tlx = t_lx > 0 ? t_lx : p->g.lx;
    p->tly = t_ly > 0 ? t_ly : p->g.ly;
    if (dT_dev != p->tmap)
        SHG_CK(cudaMemcpyAsync(p->tmap, dT_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    SHG_CK(launch_build_ttab(p->fp64, p->tmap, p->ttab, tx, ty, tz, p->c.L / (tz - 1),
                             plan_dk_model(p), s));
    // per-point table (FP32): tz layers of the field grid
    const size_t ub = size_t(tz) * p->g.nx * p->g.ny * sizeof(float2);
    const bool want = !p->fp64 && !(p->flags & SHG_FLAG_NODE_SAMPLER) && ub <= kUmapMaxBytes &&
                      tz <= 65535;
    if (p->umap && (!want || p->umap_bytes != ub)) {
        cudaFree(p->umap);
        p->umap = nullptr;
        p->umap_bytes = 0;
    }
    if (want && !p->umap) {
        SHG_CK(cudaMalloc(&p->umap, ub));
        p->umap_bytes = ub;
    }
    SHG_CK(cudaStreamSynchronize(s));
    shg_status_t r = upload_desc(p);
    if (r != SHG_OK || !p->umap) return r;
    SHG_CK(launch_upsample_map(p->desc, p->umap, p->g.nx, p->g.ny, tz, s));
    SHG_CK(cudaStreamSynchronize(s));
    return SHG_OK;
}

shg_status_t shg_set_temperature_batch(shg_plan_t* const* plans, int n, const float* const* dT_devs,
                                       int tx, int ty, int tz, const double* t_lx,
                                       const double* t_ly, shg_stream_t stream) {
    if (!plans || n <= 0 || !dT_devs || !t_lx || !t_ly || !distinct_plans(plans, n))
        return SHG_ERR_INVALID_ARG;
    // all arguments of all plans are checked before any plan changes, so a
    // refused call leaves every plan's map as it was
    if (tx < 2 || ty < 2 || tz < 2) return SHG_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!plans[k] || !dT_devs[k] || !std::isfinite(t_lx[k]) || !std::isfinite(t_ly[k]))
            return SHG_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // plans whose installed map has this shape and extent are rebuilt together;
    // the others take the single-plan path (which may allocate and synchronise)
    std::vector<int> fast;
    for (int k = 0; k < n; ++k) {
        shg_plan* p = plans[k];
        const bool same = p->ttab != nullptr && p->tx == tx && p->ty == ty && p->tz == tz &&
                          p->tlx == (t_lx[k] > 0 ? t_lx[k] : p->g.lx) &&
                          p->tly == (t_ly[k] > 0 ? t_ly[k] : p->g.ly);
        if (same) {
            fast.push_back(k);
        } else {
            const shg_status_t r = shg_set_temperature(p, dT_devs[k], tx, ty, tz, t_lx[k],
                                                       t_ly[k], stream);
            if (r != SHG_OK) return r;
        }
    }
    if (fast.empty()) return SHG_OK;
    for (int k : fast) {
        adjoint_forward_state(plans[k], false);
        if (plans[k]->done_valid) SHG_CK(cudaStreamWaitEvent(s, plans[k]->done, 0));
        if (plans[k]->ready_pending) SHG_CK(cudaStreamWaitEvent(s, plans[k]->ready, 0));
    }
    // (dT, C) tables, one launch per precision
    for (int prec = 0; prec < 2; ++prec) {
        std::vector<TtabJob> jobs;
        for (int k : fast) {
            shg_plan* p = plans[k];
            if (p->fp64 != (prec == 1)) continue;
            jobs.push_back(TtabJob{dT_devs[k], p->tmap, p->ttab, p->c.L / (tz - 1),
                                   plan_dk_model(p)});
        }
        if (jobs.empty()) continue;
        void* dj = nullptr;
        SHG_CK(cudaMallocAsync(&dj, jobs.size() * sizeof(TtabJob), s));
        SHG_CK(cudaMemcpyAsync(dj, jobs.data(), jobs.size() * sizeof(TtabJob),
                               cudaMemcpyHostToDevice, s));
        SHG_CK(launch_build_ttab_batch(prec == 1, static_cast<const TtabJob*>(dj), int(jobs.size()),
                                       tx, ty, tz, s));
        SHG_CK(cudaFreeAsync(dj, s));
    }
    // per-point tables, one launch per grid
    std::map<std::pair<int, int>, std::vector<int>> grids;
    for (int k : fast)
        if (plans[k]->umap) grids[{plans[k]->g.nx, plans[k]->g.ny}].push_back(k);
    for (auto& kv : grids) {
        const std::vector<int>& ks = kv.second;
        const int chunk = std::max(1, 65535 / tz);
        for (size_t b = 0; b < ks.size(); b += chunk) {
            const size_t m = std::min(ks.size() - b, size_t(chunk));
            std::vector<const void*> ptrs(2 * m);
            for (size_t i = 0; i < m; ++i) {
                ptrs[i] = plans[ks[b + i]]->desc;
                ptrs[m + i] = plans[ks[b + i]]->umap;
            }
            void* dp = nullptr;
            SHG_CK(cudaMallocAsync(&dp, ptrs.size() * sizeof(void*), s));
            SHG_CK(cudaMemcpyAsync(dp, ptrs.data(), ptrs.size() * sizeof(void*),
                                   cudaMemcpyHostToDevice, s));
            void* const* dv = static_cast<void* const*>(dp);
            SHG_CK(launch_upsample_map_batch(reinterpret_cast<const void* const*>(dv), dv + m,
                                             int(m), kv.first.first, kv.first.second, tz, s));
            SHG_CK(cudaFreeAsync(dp, s));
        }
    }
    for (int k : fast) {
        SHG_CK(cudaEventRecord(plans[k]->ready, s));
        plans[k]->ready_pending = true;
    }
    return SHG_OK;
}

shg_status_t shg_set_fields(shg_plan_t* p, const void* a_f_dev, const void* a_sh_dev,
                            shg_stream_t stream) {
    if (!p || p->w3) return SHG_ERR_INVALID_ARG;
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    adjoint_forward_state(p, false);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t one = size_t(p->g.nx) * p->g.ny * p->csize;
    if (!p->field0) SHG_CK(cudaMalloc(&p->field0, 2 * one));
    unsigned char* f0 = static_cast<unsigned char*>(p->field0);
    if (a_f_dev)
        SHG_CK(cudaMemcpyAsync(f0, a_f_dev, one, cudaMemcpyDeviceToDevice, s));
    else
        SHG_CK(cudaMemsetAsync(f0, 0, one, s));
    if (a_sh_dev)
        SHG_CK(cudaMemcpyAsync(f0 + one, a_sh_dev, one, cudaMemcpyDeviceToDevice, s));
    else
        SHG_CK(cudaMemsetAsync(f0 + one, 0, one, s));
    SHG_CK(cudaStreamSynchronize(s));
    if (!p->custom_init) p->gvalid = false;
    p->custom_init = true;
    return upload_desc(p);
}

shg_status_t shg_propagate(shg_plan_t* p, shg_stream_t stream) {
    if (!p) return SHG_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->ready_pending) SHG_CK(cudaStreamWaitEvent(s, p->ready, 0));
    shg_status_t st = plan_forward(p, s);
    if (st != SHG_OK) return st;
    adjoint_forward_state(p, true);
    SHG_CK(cudaEventRecord(p->done, s));
    p->done_valid = true;
    p->has_result = true;
    p->batch_result = false;
    p->last_stream = s;
    return SHG_OK;
}

shg_status_t shg_efficiency(shg_plan_t* p, double* eta, double* p_f, double* p_sh) {
    if (!p) return SHG_ERR_INVALID_ARG;
    if (!p->has_result) return SHG_ERR_STATE;
    if (p->w3) {
        double pw[3];
        shg_status_t r = three_wave_powers(p, pw);
        if (r != SHG_OK) return r;
        const double pin = three_wave_input_power(p);
        const double e = pin > 0 ? pw[2] / pin : 0.0;
        if (eta) *eta = e;
        if (p_f) *p_f = pw[0];
        if (p_sh) *p_sh = pw[2];
        return (std::isfinite(e) && std::isfinite(pw[0]) && std::isfinite(pw[1])) ? SHG_OK
                                                                                  : SHG_ERR_NONFINITE;
    }
    SHG_CK(cudaStreamSynchronize(p->last_stream));
    int kst = p->batch_kst;  // a batch reports kernel errors per instance on the host
    if (!p->batch_result)
        SHG_CK(cudaMemcpy(&kst, p->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (kst != 0) return shg_status_t(kst);
    if (!p->batch_result)
        SHG_CK(cudaMemcpy(p->pw_host, p->pw, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    const double e = p->b.p1 > 0 ? p->pw_host[1] / p->b.p1 : 0.0;
    if (eta) *eta = e;
    if (p_f) *p_f = p->pw_host[0];
    if (p_sh) *p_sh = p->pw_host[1];
    if (!std::isfinite(e) || !std::isfinite(p->pw_host[0])) return SHG_ERR_NONFINITE;
    return SHG_OK;
}

shg_status_t shg_get_fields(shg_plan_t* p, void* a_f_dev, void* a_sh_dev, shg_stream_t stream) {
    if (!p || p->w3) return SHG_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->last_stream != s && p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    const size_t one = size_t(p->g.nx) * p->g.ny * p->csize;
    const unsigned char* f = static_cast<const unsigned char*>(p->field);
    if (a_f_dev) SHG_CK(cudaMemcpyAsync(a_f_dev, f, one, cudaMemcpyDeviceToDevice, s));
    if (a_sh_dev) SHG_CK(cudaMemcpyAsync(a_sh_dev, f + one, one, cudaMemcpyDeviceToDevice, s));
    return SHG_OK;
}

shg_status_t shg_get_field(shg_plan_t* p, int j, void* dev, shg_stream_t stream) {
    const int nf = (p && p->w3) ? 3 : 2;
    if (!p || !dev || j < 0 || j >= nf) return SHG_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->last_stream != s && p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    const size_t one = size_t(p->g.nx) * p->g.ny * p->csize;
    SHG_CK(cudaMemcpyAsync(dev, static_cast<const unsigned char*>(p->field) + size_t(j) * one, one,
                           cudaMemcpyDeviceToDevice, s));
    return SHG_OK;
}

shg_status_t shg_powers(shg_plan_t* p, double* out, int n) {
    const int nf = (p && p->w3) ? 3 : 2;
    if (!p || !out || n < nf) return SHG_ERR_INVALID_ARG;
    if (!p->has_result) return SHG_ERR_STATE;
    if (p->w3) return three_wave_powers(p, out);
    double e = 0;
    shg_status_t r = shg_efficiency(p, &e, &out[0], &out[1]);
    return r;
}

static bool finite3(const shg_crystal3_t* c, const shg_beams3_t* b) {
    const double v[] = {c->L, c->lambda1, c->lambda2, c->n1, c->n2, c->n3, c->d_eff, c->alpha[0],
                        c->alpha[1], c->alpha[2], c->beta[0], c->beta[1], c->beta[2], c->dk0,
                        c->ddk_dT, c->dn_dT, c->walkoff[0], c->walkoff[1], c->walkoff[2],
                        b->p[0], b->p[1], b->p[2], b->w0[0], b->w0[1], b->w0[2], b->z_focus[0],
                        b->z_focus[1], b->z_focus[2], b->t_oven_offset};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

shg_status_t shg_plan_create_3w(const shg_grid_t* grid, const shg_crystal3_t* c,
                                const shg_beams3_t* b, int flags, shg_plan_t** out) {
    if (out) *out = nullptr;
    if (!grid || !c || !b || !out || !finite3(c, b)) return SHG_ERR_INVALID_ARG;
    if (flags & ~SHG_FLAG_FP64) return SHG_ERR_INVALID_ARG;  // no heat grid, adjoint or sampler flags
    if (!(c->L > 0) || !(c->lambda1 > 0) || !(c->lambda2 > 0) || !(c->n1 > 0) || !(c->n2 > 0) ||
        !(c->n3 > 0))
        return SHG_ERR_INVALID_ARG;
    for (int j = 0; j < 3; ++j)
        if (!(b->w0[j] > 0) || b->p[j] < 0 || !(std::fabs(c->walkoff[j]) < 1.5))
            return SHG_ERR_INVALID_ARG;
    if (!(b->p[0] + b->p[1] + b->p[2] > 0)) return SHG_ERR_INVALID_ARG;
    // the shared state (grid checks, phase and twiddle tables, map machinery,
    // streams and events) of an SHG plan with the same grid, crystal length,
    // phase and temperature coefficients; the fields and K-space tables are
    // then replaced by three-wave ones
    shg_crystal_t c2{};
    c2.L = c->L;
    c2.lambda_f = c->lambda1;
    c2.n_f = c->n1;
    c2.n_sh = c->n3;
    c2.d_eff = c->d_eff;
    c2.dk0 = c->dk0;
    c2.ddk_dT = c->ddk_dT;
    c2.dn_dT = c->dn_dT;
    c2.kappa_th = 1.0;
    c2.wx = c2.wy = 1.0;
    shg_beams_t b2{};
    b2.p1 = b->p[0] + b->p[1] + b->p[2];
    b2.w0 = b->w0[0];
    b2.z_focus = b->z_focus[0];
    b2.t_oven_offset = b->t_oven_offset;
    b2.undepleted = b->undepleted;
    // FP32 square grids with a cluster-resident kernel read the map through the
    // per-point table; the streaming three-wave passes sample it at its nodes
    // (cluster3_size also sets that kernel's attributes, outside any capture)
    const bool c3 = !(flags & SHG_FLAG_FP64) && grid->nx == grid->ny && cluster3_size(grid->nx) > 0;
    shg_plan_t* p = nullptr;
    shg_status_t st =
        shg_plan_create(grid, &c2, &b2, flags | (c3 ? 0 : SHG_FLAG_NODE_SAMPLER), &p);
    if (st != SHG_OK) return st;
    auto fail = [&](shg_status_t s2) {
        shg_plan_destroy(p);
        return s2;
    };
    const size_t npts = size_t(grid->nx) * grid->ny;
    cudaFree(p->field);
    cudaFree(p->px);
    cudaFree(p->py);
    p->field = p->px = p->py = nullptr;
    if (p->cmap_dev) cudaFree(p->cmap_dev);  // the tensor map described the two-field buffer
    p->cmap_dev = nullptr;
    p->has_cmap = false;
    cudaError_t e;
    if ((e = cudaMalloc(&p->field, 3 * npts * p->csize)) != cudaSuccess ||
        (e = cudaMemset(p->field, 0, 3 * npts * p->csize)) != cudaSuccess ||
        (e = cudaMalloc(&p->px, size_t(3) * grid->nx * 16)) != cudaSuccess ||
        (e = cudaMalloc(&p->py, size_t(3) * grid->ny * 16)) != cudaSuccess)
        return fail(cuda_fail(e, "three-wave buffers"));
    if ((st = three_wave_alloc(p, c, b)) != SHG_OK || (st = build_prop_tables3(p, p->px, p->py)) != SHG_OK ||
        (st = upload_desc(p)) != SHG_OK)
        return fail(st);
    *out = p;
    return SHG_OK;
}

shg_status_t shg_set_monitor(shg_plan_t* p, int every) {
    if (!p || every < 0 || p->w3) return SHG_ERR_INVALID_ARG;
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    if (p->mon) {
        cudaFree(p->mon);
        p->mon = nullptr;
    }
    p->mon_every = 0;
    p->mon_slots = 0;
    if (every > 0) {
        const int nz = p->g.nz;
        const int slots = nz / every + 1 + (nz % every != 0 ? 1 : 0);
        SHG_CK(cudaMalloc((void**)&p->mon, 2 * size_t(slots) * sizeof(double)));
        SHG_CK(cudaMemset(p->mon, 0, 2 * size_t(slots) * sizeof(double)));
        p->mon_every = every;
        p->mon_slots = slots;
    }
    // captured graphs hold the old monitor buffer (its memset node)
    p->gvalid = false;
    forget_plan_batches(p);
    p->has_result = false;
    return upload_desc(p);
}

shg_status_t shg_set_phase_model(shg_plan_t* p, const shg_qpm_t* m) {
    if (!p || p->w3) return SHG_ERR_INVALID_ARG;
    DkModel d{};
    if (m) {
        const double v[] = {m->t_oven, m->lambda25, m->a_lambda, m->b_lambda, m->n_f[0], m->n_f[1],
                            m->n_f[2], m->n_f[3], m->n_sh[0], m->n_sh[1], m->n_sh[2], m->n_sh[3]};
        for (double x : v)
            if (!std::isfinite(x)) return SHG_ERR_INVALID_ARG;
        if (!(m->lambda25 > 0)) return SHG_ERR_INVALID_ARG;
        d.on = 1;
        d.t_oven = m->t_oven;
        d.k_mat = 4 * kPi / p->c.lambda_f;
        d.lam25 = m->lambda25;
        d.a = m->a_lambda;
        d.b = m->b_lambda;
        for (int k = 0; k < 4; ++k) {
            d.nF[k] = m->n_f[k];
            d.nS[k] = m->n_sh[k];
        }
    }
    shg_status_t st = quiesce(p);
    if (st != SHG_OK) return st;
    if (p->ready_pending) {
        SHG_CK(cudaEventSynchronize(p->ready));
        p->ready_pending = false;
    }
    adjoint_forward_state(p, false);
    const bool was_on = p->dkm.on != 0;
    p->dkm = d;
    if ((st = build_phase_table(p)) != SHG_OK) return st;
    if ((st = upload_desc(p)) != SHG_OK) return st;
    if (p->ttab && (d.on || was_on)) {
        // the map's C channel changes meaning: rebuild it from the stored map
        SHG_CK(launch_build_ttab(p->fp64, p->tmap, p->ttab, p->tx, p->ty, p->tz,
                                 p->c.L / (p->tz - 1), plan_dk_model(p), nullptr));
        if (p->umap)
            SHG_CK(launch_upsample_map(p->desc, p->umap, p->g.nx, p->g.ny, p->tz, nullptr));
        SHG_CK(cudaStreamSynchronize(nullptr));
    }
    return SHG_OK;
}

shg_status_t shg_get_monitor(shg_plan_t* p, double* z_out, double* p_f_out, double* p_sh_out,
                             int max_samples, int* n_samples) {
    if (!p || max_samples < 0) return SHG_ERR_INVALID_ARG;
    if (!p->mon || !p->has_result) return SHG_ERR_STATE;
    SHG_CK(cudaStreamSynchronize(p->last_stream));
    std::vector<double> h(2 * size_t(p->mon_slots));
    SHG_CK(cudaMemcpy(h.data(), p->mon, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    const double dxdy = (p->g.lx / p->g.nx) * (p->g.ly / p->g.ny);
    const double cF = 0.5 * kEps0 * kCLight * p->c.n_f * dxdy;
    const double cS = 0.5 * kEps0 * kCLight * p->c.n_sh * dxdy;
    const double dz = p->c.L / p->g.nz;
    const int n = std::min(max_samples, p->mon_slots);
    bool finite = true;
    for (int m = 0; m < n; ++m) {
        const bool last = (m == p->mon_slots - 1);
        const int s = last ? p->g.nz : m * p->mon_every;
        if (z_out) z_out[m] = s * dz;
        if (p_f_out) p_f_out[m] = cF * h[2 * m];
        if (p_sh_out) p_sh_out[m] = cS * h[2 * m + 1];
        finite &= std::isfinite(h[2 * m]) && std::isfinite(h[2 * m + 1]);
    }
    if (n_samples) *n_samples = p->mon_slots;
    return finite ? SHG_OK : SHG_ERR_NONFINITE;
}

}  // extern "C"

// ============================================================ batches ====

namespace shg {

struct BatchGroup {
    bool fp64;
    int nx, ny, nz;
    bool custom;
    int row_bits = 0;           // row_umap_bit() of the plans when the graph was captured
    std::vector<shg_plan*> plans;
    std::vector<int> index;     // position of each plan in the caller's list
    void* descs = nullptr;      // device InstDesc[n]
    InitDesc* idescs = nullptr; // device InitDesc[n]
    double* pw = nullptr;       // device [n][2]
    int* status = nullptr;      // device [n]: the instances' status words during a batch
    void* tmaps = nullptr;      // device CUtensorMap[n], or nullptr (cp.async column pass)
    size_t off = 0;             // first instance of the group in the entry's staging arrays
    unsigned char* hdesc = nullptr;  // pinned staging of the descriptors [n]
    InitDesc* hinit = nullptr;       // pinned staging of the init descriptors [n]
};

struct BatchEntry {
    std::vector<BatchGroup> groups;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    double* pw_host = nullptr;  // pinned [n][2], the caller's order
    double* pw_stage = nullptr; // pinned [n][2], group order (one copy per group)
    int* st_stage = nullptr;    // pinned [n], group order
    cudaEvent_t uploaded = nullptr;  // after the last descriptor upload from the staging
    int n = 0;
    bool valid = false;
};

static std::mutex g_batch_mu;
static std::map<std::vector<shg_plan*>, BatchEntry*> g_batches;

static void free_entry(BatchEntry* b) {
    // the staging buffers may still be read by an upload in flight
    if (b->uploaded) cudaEventSynchronize(b->uploaded);
    for (auto& g : b->groups) {
        if (g.descs) cudaFree(g.descs);
        if (g.idescs) cudaFree(g.idescs);
        if (g.pw) cudaFree(g.pw);
        if (g.status) cudaFree(g.status);
        if (g.tmaps) cudaFree(g.tmaps);
        if (g.hdesc) cudaFreeHost(g.hdesc);
        if (g.hinit) cudaFreeHost(g.hinit);
    }
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto s : b->side) cudaStreamDestroy(s);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->pw_host) cudaFreeHost(b->pw_host);
    if (b->pw_stage) cudaFreeHost(b->pw_stage);
    if (b->st_stage) cudaFreeHost(b->st_stage);
    if (b->uploaded) cudaEventDestroy(b->uploaded);
    delete b;
}

static shg_status_t build_entry(const std::vector<shg_plan*>& plans, BatchEntry** out) {
    BatchEntry* b = new BatchEntry();
    b->n = int(plans.size());
    for (int i = 0; i < b->n; ++i) {
        shg_plan* p = plans[i];
        BatchGroup* g = nullptr;
        for (auto& gg : b->groups)
            if (gg.fp64 == p->fp64 && gg.nx == p->g.nx && gg.ny == p->g.ny && gg.nz == p->g.nz &&
                gg.custom == p->custom_init)
                g = &gg;
        if (!g) {
            b->groups.push_back(BatchGroup{p->fp64, p->g.nx, p->g.ny, p->g.nz, p->custom_init});
            g = &b->groups.back();
        }
        g->plans.push_back(p);
        g->index.push_back(i);
    }
    for (auto& g : b->groups) g.row_bits = row_umap_bit(g.plans);
    cudaError_t e;
    for (auto& g : b->groups) {
        const int n = int(g.plans.size());
        if ((e = cudaMalloc(&g.descs, n * desc_bytes(g.fp64))) != cudaSuccess ||
            (e = cudaMalloc((void**)&g.idescs, n * sizeof(InitDesc))) != cudaSuccess ||
            (e = cudaMalloc((void**)&g.pw, n * 2 * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&g.status, n * sizeof(int))) != cudaSuccess ||
            (e = cudaMallocHost((void**)&g.hdesc, n * desc_bytes(g.fp64))) != cudaSuccess ||
            (e = cudaMallocHost((void**)&g.hinit, n * sizeof(InitDesc))) != cudaSuccess) {
            free_entry(b);
            return cuda_fail(e, "batch alloc");
        }
        bool all_tmaps = true;
        for (shg_plan* p : g.plans) all_tmaps &= p->has_cmap;
        if (all_tmaps) {
            std::vector<CUtensorMap> hm(n);
            for (int k = 0; k < n; ++k) hm[k] = g.plans[k]->cmap;
            if ((e = cudaMalloc(&g.tmaps, n * sizeof(CUtensorMap))) != cudaSuccess ||
                (e = cudaMemcpy(g.tmaps, hm.data(), n * sizeof(CUtensorMap),
                                cudaMemcpyHostToDevice)) != cudaSuccess) {
                free_entry(b);
                return cuda_fail(e, "batch tensor maps");
            }
        }
    }
    size_t off = 0;
    for (auto& g : b->groups) {
        g.off = off;
        off += g.plans.size();
    }
    if ((e = cudaMallocHost((void**)&b->pw_host, b->n * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&b->pw_stage, b->n * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&b->st_stage, b->n * sizeof(int))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        free_entry(b);
        return cuda_fail(e, "batch setup");
    }
    for (size_t i = 0; i < b->groups.size(); ++i) {
        cudaStream_t s;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            free_entry(b);
            return cuda_fail(e, "batch streams");
        }
        b->side.push_back(s);
        b->ev.push_back(ev);
    }
    cudaEvent_t fork;
    if ((e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess) {
        free_entry(b);
        return cuda_fail(e, "batch event");
    }
    b->ev.push_back(fork);
    *out = b;
    return SHG_OK;
}

// Upload the current descriptors of every plan of the entry, from pinned
// staging buffers owned by the entry (so the copies need no host wait; the
// next refresh reuses the staging only after the previous submit has
// synchronised its stream).  Inside a batch every instance reports kernel
// errors into its slot of the group's status array, which one copy reads.
static shg_status_t refresh_entry(BatchEntry* b, cudaStream_t st) {
    for (auto& g : b->groups) {
        const int n = int(g.plans.size());
        const size_t db = desc_bytes(g.fp64);
        for (int k = 0; k < n; ++k) {
            unsigned char* d = g.hdesc + k * db;
            fill_desc_any(g.plans[k], d);
            if (g.fp64)
                reinterpret_cast<InstDesc<double>*>(d)->status = g.status + k;
            else
                reinterpret_cast<InstDesc<float>*>(d)->status = g.status + k;
            fill_init(g.plans[k], &g.hinit[k]);
            g.hinit[k].pw = g.pw + 2 * k;
        }
        SHG_CK(cudaMemcpyAsync(g.descs, g.hdesc, n * db, cudaMemcpyHostToDevice, st));
        SHG_CK(cudaMemcpyAsync(g.idescs, g.hinit, n * sizeof(InitDesc), cudaMemcpyHostToDevice,
                               st));
    }
    SHG_CK(cudaEventRecord(b->uploaded, st));
    return SHG_OK;
}

static shg_status_t enqueue_batch(BatchEntry* b, cudaStream_t st) {
    // fork the groups onto side streams so that instances of different grids
    // overlap, then join
    const int ng = int(b->groups.size());
    PdlScope pdl(ng == 1);
    // the group with the most point-steps launches at the highest priority
    int lowest = 0, highest = 0;
    SHG_CK(cudaDeviceGetStreamPriorityRange(&lowest, &highest));
    int big = 0;
    double w_big = -1;
    for (int i = 0; i < ng; ++i) {
        const BatchGroup& g = b->groups[i];
        const double w = double(g.nx) * g.ny * g.nz * double(g.plans.size());
        if (w > w_big) {
            w_big = w;
            big = i;
        }
    }
    cudaEvent_t fork = b->ev.back();
    SHG_CK(cudaEventRecord(fork, st));
    for (int i = 0; i < ng; ++i) {
        BatchGroup& g = b->groups[i];
        cudaStream_t s = b->side[i];
        SHG_CK(cudaStreamWaitEvent(s, fork, 0));
        launch_priority = (ng > 1 && i == big) ? highest : 0;
        shg_status_t r = enqueue_forward(g.fp64, g.nx, g.ny, g.nz, g.descs, g.idescs,
                                         int(g.plans.size()), g.plans[0]->tw, g.plans, s, g.tmaps,
                                         g.status);
        launch_priority = 0;
        if (r != SHG_OK) return r;
        SHG_CK(cudaEventRecord(b->ev[i], s));
        SHG_CK(cudaStreamWaitEvent(st, b->ev[i], 0));
    }
    return SHG_OK;
}

}  // namespace shg

namespace shg {
void forget_plan_batches(shg_plan* p) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        bool has = false;
        for (auto q : it->first) has |= (q == p);
        if (has) {
            free_entry(it->second);
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}
}  // namespace shg

extern "C" shg_status_t shg_batch_submit(shg_plan_t* const* plans, int n, double* eta_host_out,
                                         shg_stream_t stream) {
    if (!plans || n <= 0 || !distinct_plans(plans, n)) return SHG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (plans[i]->w3) return SHG_ERR_INVALID_ARG;  // three-wave plans propagate one by one
    std::vector<shg_plan*> key(plans, plans + n);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchEntry*& ent = g_batches[key];
    shg_status_t r;
    if (ent) {
        // the captured graph depends on each plan's init kind; rebuild if changed
        bool stale = false;
        for (auto& g : ent->groups) {
            for (auto p : g.plans) stale |= (p->custom_init != g.custom);
            stale |= row_umap_bit(g.plans) != g.row_bits;
        }
        if (stale) {
            free_entry(ent);
            ent = nullptr;
        }
    }
    if (!ent) {
        if ((r = build_entry(key, &ent)) != SHG_OK) {
            g_batches.erase(key);
            return r;
        }
    }
    for (auto p : key) {
        if (p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
        if (p->ready_pending) SHG_CK(cudaStreamWaitEvent(st, p->ready, 0));
    }
    if ((r = refresh_entry(ent, st)) != SHG_OK) return r;
    for (auto& g : ent->groups) {
        int hx = 0, hy = 0;
        for (shg_plan* p : g.plans)
            if ((p->flags & SHG_FLAG_THERMAL) && p->Q) {
                hx = std::max(hx, p->g.hx);
                hy = std::max(hy, p->g.hy);
            }
        const int rb = row_umap_bit(g.plans);
        if ((r = tune_group(g.fp64, g.nx, g.ny, g.nz, g.descs, int(g.plans.size()),
                            g.plans[0]->tw, hx, st, g.tmaps, rb,
                            step_schedule(g.fp64, g.plans, rb), hy)) != SHG_OK)
            return r;
    }
    if (use_graphs()) {
        if (!ent->valid) {
            if (ent->gexec) {
                cudaGraphExecDestroy(ent->gexec);
                ent->gexec = nullptr;
            }
            r = capture(ent->cap, [&](cudaStream_t s) { return enqueue_batch(ent, s); },
                        &ent->gexec);
            if (r != SHG_OK) return r;
            ent->valid = true;
        }
        SHG_CK(cudaGraphLaunch(ent->gexec, st));
    } else {
        if ((r = enqueue_batch(ent, st)) != SHG_OK) return r;
    }
    // gather the powers and the status words: one copy of each per group
    for (auto& g : ent->groups) {
        const size_t m = g.plans.size();
        SHG_CK(cudaMemcpyAsync(ent->pw_stage + 2 * g.off, g.pw, 2 * m * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaMemcpyAsync(ent->st_stage + g.off, g.status, m * sizeof(int),
                               cudaMemcpyDeviceToHost, st));
    }
    SHG_CK(cudaStreamSynchronize(st));
    int first_err = 0;
    for (auto& g : ent->groups)
        for (size_t k = 0; k < g.plans.size(); ++k) {
            const int i = g.index[k];
            ent->pw_host[2 * i] = ent->pw_stage[2 * (g.off + k)];
            ent->pw_host[2 * i + 1] = ent->pw_stage[2 * (g.off + k) + 1];
            const int kst = ent->st_stage[g.off + k];
            g.plans[k]->batch_kst = kst;
            if (kst != 0 && first_err == 0) first_err = kst;
        }
    if (first_err != 0) {
        for (auto p : key) {
            adjoint_forward_state(p, false);  // the checkpoints of a failed sweep are unusable
            p->last_stream = st;
            p->has_result = true;
            p->batch_result = true;
            p->ready_pending = false;
            p->done_valid = false;
        }
        return shg_status_t(first_err);
    }
    bool finite = true;
    for (int i = 0; i < n; ++i) {
        shg_plan* p = key[i];
        p->pw_host[0] = ent->pw_host[2 * i];
        p->pw_host[1] = ent->pw_host[2 * i + 1];
        const double e = p->b.p1 > 0 ? p->pw_host[1] / p->b.p1 : 0.0;
        if (eta_host_out) eta_host_out[i] = e;
        finite &= std::isfinite(e);
        p->last_stream = st;
        p->has_result = true;
        p->batch_result = true;
        adjoint_forward_state(p, true);  // the batch wrote its checkpoints too
        p->ready_pending = false;  // the batch waited for it and has completed
        p->done_valid = false;
    }
    return finite ? SHG_OK : SHG_ERR_NONFINITE;
}

extern "C" shg_status_t shg_pass_times(shg_plan_t* const* plans, int n, int nsteps, double* out,
                                       int* inst_out, int max_groups, int* ngroups,
                                       shg_stream_t stream) {
    if (!plans || n <= 0 || nsteps <= 0 || !out || !ngroups || max_groups <= 0 ||
        !distinct_plans(plans, n))
        return SHG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (plans[i]->w3) return SHG_ERR_INVALID_ARG;
    std::vector<shg_plan*> key(plans, plans + n);
    for (auto p : key)
        if (!p) return SHG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n; ++i)
        if (plans[i] && plans[i]->ready_pending) SHG_CK(cudaStreamWaitEvent(st, plans[i]->ready, 0));
    BatchEntry* ent = nullptr;
    shg_status_t r = build_entry(key, &ent);
    if (r != SHG_OK) return r;
    if ((r = refresh_entry(ent, st)) != SHG_OK) {
        free_entry(ent);
        return r;
    }
    const int ng = int(ent->groups.size());
    if (ng > max_groups) {
        free_entry(ent);
        return SHG_ERR_INVALID_ARG;
    }
    std::vector<cudaEvent_t> ev(4 * nsteps * ng, nullptr);
    std::vector<int> one_pass(ng, 0);
    auto release = [&] {
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
        free_entry(ent);
    };
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    for (int s = 1; s <= nsteps && e == cudaSuccess; ++s) {
        for (int gi = 0; gi < ng && e == cudaSuccess; ++gi) {
            BatchGroup& g = ent->groups[gi];
            const int zs = std::min(s, g.nz - 1 > 0 ? g.nz - 1 : 0);
            cudaEvent_t* E = &ev[4 * ((s - 1) * ng + gi)];
            cudaEventRecord(E[0], st);
            int hx = 0, hy = 0;
            for (shg_plan* p : g.plans)
                if ((p->flags & SHG_FLAG_THERMAL) && p->Q) {
                    hx = std::max(hx, p->g.hx);
                    hy = std::max(hy, p->g.hy);
                }
            if (s == 1) {
                const int rb0 = row_umap_bit(g.plans);
                shg_status_t r2 = tune_group(g.fp64, g.nx, g.ny, g.nz, g.descs,
                                             int(g.plans.size()), g.plans[0]->tw, hx, st, g.tmaps,
                                             rb0, step_schedule(g.fp64, g.plans, rb0), hy);
                if (r2 != SHG_OK) {
                    release();
                    return r2;
                }
                cudaEventRecord(E[0], st);
            }
            const int rbg = row_umap_bit(g.plans);
            const int vrg = fft_variant(g.fp64, g.nx, 0, rbg, int(g.plans.size())) | rbg;
            // the kernels the group's propagation runs: with one pass per step,
            // a row-layout pass (s = 2) and a column-layout pass (s = 1)
            const bool steps = step_schedule(g.fp64, g.plans, rbg) && g.nz >= 3;
            one_pass[gi] = steps ? 1 : 0;
            if (steps)
                e = launch_row_step(g.nx, g.descs, int(g.plans.size()), g.ny, g.nz, 2,
                                    g.plans[0]->tw, hx, st,
                                    step_variant(g.fp64, g.nx, 0, int(g.plans.size())) | rbg);
            else
                e = launch_row(g.fp64, g.nx, g.descs, int(g.plans.size()), g.ny, g.nz, zs,
                               g.plans[0]->tw, hx, st, vrg);
            cudaEventRecord(E[1], st);
            if (e == cudaSuccess) {
                cudaEventRecord(E[2], st);
                if (steps)
                    e = launch_col_step(g.ny, g.descs, int(g.plans.size()), g.nx, g.nz, 1,
                                        g.plans[0]->tw, hy, st,
                                        step_variant(g.fp64, g.ny, 1, int(g.plans.size())));
                else
                    e = launch_col(g.fp64, g.ny, g.descs, int(g.plans.size()), g.nx,
                                   g.plans[0]->tw, st,
                                   fft_variant(g.fp64, g.ny, 1, 0, int(g.plans.size())), g.tmaps);
                cudaEventRecord(E[3], st);
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        for (int gi = 0; gi < ng; ++gi) {
            double tr = 0, tc = 0;
            for (int s = 0; s < nsteps; ++s) {
                cudaEvent_t* E = &ev[4 * (s * ng + gi)];
                float a = 0, b = 0;
                cudaEventElapsedTime(&a, E[0], E[1]);
                cudaEventElapsedTime(&b, E[2], E[3]);
                tr += a;
                tc += b;
            }
            out[5 * gi] = ent->groups[gi].nx;
            out[5 * gi + 1] = ent->groups[gi].ny;
            out[5 * gi + 2] = tr / nsteps;
            out[5 * gi + 3] = tc / nsteps;
            out[5 * gi + 4] = one_pass[gi] ? 1 : 2;
            if (inst_out) inst_out[gi] = int(ent->groups[gi].plans.size());
        }
        *ngroups = ng;
    }
    release();
    return e == cudaSuccess ? SHG_OK : cuda_fail(e, "shg_pass_times");
}
