// Host runtime behind the C ABI of include/lbm_cde.h: handle, buffers,
// parameter derivation (D -> A, Eq. 36 / A.6), ping-pong stepping, reductions,
// checkpoints. Every entry point catches its own failures and returns a status.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_cde.h"
#include "lbm_internal.cuh"

using lbm::LaunchCfg;
using lbm::StepArgs;

struct lbm_cde_s {
    lbm_cde_desc d{};
    int q = 9, dim = 2;
    long long ncell = 0;
    size_t elem = 4;
    bool neq = false;
    void* state[2] = {nullptr, nullptr};
    float* phi[2] = {nullptr, nullptr};
    float* phi_tmp = nullptr;      // host round trips (run_host)
    double* partials = nullptr;    // reduction scratch
    double* sum_dev = nullptr;
    int nparts = 0;
    int cur = 0;
    lbm::Coef coef{};
    double A[9] = {0};
    double s[15] = {0};
    double alpha1 = 0, alpha2 = 0;
    bool d_set = false;
    int ukind = LBM_U_NONE;
    const float* ua = nullptr;
    const float* sched = nullptr;
    long long sched_len = 0;
    long long t = 0;
    bool ready = false;
    LaunchCfg cfg{256, 1};
    cudaStream_t st = nullptr;
    std::string err;
    // adjoint: checkpoints of the forward run, segment recompute buffer, adjoint states
    std::vector<void*> ck;
    int64_t ck_every = 0, ck_nsteps = 0;
    void* seg = nullptr;           // recomputed states of a checkpoint segment
    void* seg2 = nullptr;          // second segment buffer (overlapped reverse sweep), or NULL
    int64_t seg_states = 0;
    cudaStream_t st_rec = nullptr; // stream of the segment recompute in the overlapped sweep
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr}, ev_start = nullptr;
    float* mu[2] = {nullptr, nullptr};
    float* adj_partials = nullptr;
    float2* grad_acc = nullptr;
    float* phi0_saved = nullptr;
    bool have_fwd = false;
    // TMA-staged D2Q9 step (launch vec 7): tensor maps per source buffer, and the
    // device status word its bounded waits report to
    lbm::TmaMaps tmaps[2];
    bool tmaps_ok = false;
    const float* tmaps_ua = nullptr;
    int* status_dev = nullptr;
    long long wait_limit = 4000000000LL;   // SM cycles per bounded device wait (about 2 s)
    int zwalk = 0;                         // z-walk kernel: planes per CTA (0: automatic)
    int sms = 152;                         // multiprocessors of the device (adjoint grid)
    // per-phase device time of the last backward sweep (lbm_cde_set_profiling)
    bool prof = false;
    double prof_ms[3] = {0, 0, 0};
};

static thread_local std::string g_create_err;

static lbm_status fail(lbm_cde_t h, lbm_status s, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_err = msg;
    return s;
}

static lbm_status cuda_fail(lbm_cde_t h, cudaError_t e, const char* what)
{
    return fail(h, LBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                         \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #call); \
    } while (0)

static void* dev_alloc(lbm_cde_t h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (h->d.alloc) return h->d.alloc(bytes, h->d.alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free(lbm_cde_t h, void* p)
{
    if (!p) return;
    if (h->d.free_) h->d.free_(p, h->d.alloc_ctx);
    else if (!h->d.alloc) cudaFree(p);
}

// ---------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------
// The k in D = k (I - A/2) A^-1: Eq. 36 (modified S) or Eq. 29 (unmodified S
// of the MRT-B models, k = 2/3 + alpha1/24) for D2Q9, Eq. A.6 for D3Q15.
static double diffusion_factor(int q, double a1, double a2, int model = LBM_MRT_A)
{
    if (q == 9) return model == LBM_MRT_A ? 2.0 / 3.0 + a1 / 8.0 + a2 / 12.0 : 2.0 / 3.0 + a1 / 24.0;
    return 2.0 / 3.0 + 55.0 / 54.0 * a1 + a2 / 216.0;
}

// Inverse of a small dense matrix (n <= 3) by cofactors; returns false if singular.
static bool small_inverse(int n, const double* a, double* inv)
{
    if (n == 2) {
        const double det = a[0] * a[3] - a[1] * a[2];
        if (det == 0.0 || !std::isfinite(det)) return false;
        inv[0] = a[3] / det; inv[1] = -a[1] / det;
        inv[2] = -a[2] / det; inv[3] = a[0] / det;
        return true;
    }
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8],
                 c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0 || !std::isfinite(det)) return false;
    inv[0] = c00 / det;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    return true;
}

// Positive definiteness of a symmetric matrix by Cholesky.
static bool spd(int n, const double* a)
{
    double L[9] = {0};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = a[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * n + i] = std::sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    return true;
}

static void refresh_coef(lbm_cde_t h)
{
    lbm::Coef& c = h->coef;
    const int n = h->dim;
    double s[15];
    for (int k = 0; k < 15; ++k) s[k] = h->s[k];
    if (h->d.tie_q_rates) {
        s[4] = h->A[0];
        s[6] = h->A[n + 1];
        if (n == 3) s[8] = h->A[8];
    }
    for (int k = 0; k < 15; ++k) c.s[k] = (float)s[k];
    for (int k = 0; k < 9; ++k) c.A[k] = 0.f, c.C[k] = 0.f;
    const int model = h->d.model;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const double Aab = h->A[a * n + b];
            c.A[a * n + b] = (float)Aab;
            // Eq. 30a-b / A.5: coupling of flux row a to q-moment b (MRT-A only;
            // the MRT-B models use the unmodified S of Eq. 24)
            c.C[a * n + b] = model == LBM_MRT_A ? (float)((Aab / 2.0 - (a == b ? 1.0 : 0.0)) * s[4 + 2 * b]) : 0.f;
        }
    const bool quad = model == LBM_MRT_B1 || model == LBM_MRT_B2;
    c.b1 = quad ? 3.f : 0.f;
    c.b2 = quad ? -3.f : 0.f;
    c.g7 = quad ? 1.f : 0.f;
    c.g8 = c.g7;
    const double a1 = h->alpha1, a2 = h->alpha2;
    if (h->q == 9) {
        c.meq1 = (float)(a1 / 4.0);
        c.meq2 = (float)(a2 / 4.0);
        // Eq. 17
        c.w0 = (float)((-a1 + a2 + 4.0) / 36.0);
        c.wa = (float)((-a1 - 2.0 * a2 + 16.0) / 144.0);
        c.wd = (float)((2.0 * a1 + a2 + 16.0) / 144.0);
        c.ka = (float)(48.0 / 144.0);
        c.kd = (float)(12.0 / 144.0);
        lbm::fold_offset_coef(c);
    } else {
        c.meq1 = (float)(5.0 * a1 / 6.0);
        c.meq2 = (float)(a2 / 24.0);
        // f^eq = M^-1 m^eq for Eq. A.3 with c1 = 1, c2 = -4 (Eq. A.4)
        c.w0 = (float)(1.0 / 15.0 - 5.0 * a1 / 54.0 + a2 / 540.0);
        c.wa = (float)(1.0 / 15.0 - 5.0 * a1 / 108.0 - a2 / 2160.0);
        c.wd = (float)(1.0 / 15.0 + 5.0 * a1 / 108.0 + a2 / 8640.0);
        c.ka = (float)(1.0 / 5.0);
        c.kd = (float)(3.0 / 40.0);
        lbm::fold_offset_coef(c, 15);
    }
    const double na = h->q == 9 ? 4.0 : 6.0, nd = h->q == 9 ? 4.0 : 8.0;
    c.eps0 = (float)((double)c.w0 + na * (double)c.wa + nd * (double)c.wd - 1.0);
}

static StepArgs make_args(lbm_cde_t h, int src_idx)
{
    StepArgs a{};
    a.src = h->state[src_idx];
    a.dst = h->state[1 - src_idx];
    a.phi_src = h->phi[src_idx];
    a.phi_dst = h->phi[1 - src_idx];
    a.ua = h->ua;
    a.sched = h->sched;
    a.sched_len = h->sched_len;
    set_step(a, h->t + 1);
    a.nx = (int)h->d.nx;
    a.ny = (int)h->d.ny;
    a.nz = (int)h->d.nz;
    a.ncell = h->ncell;
    a.bc_lo = h->d.bc_lo_y;
    a.bc_hi = h->d.bc_hi_y;
    a.phiw_lo = (float)h->d.phi_w_lo_y;
    a.phiw_hi = (float)h->d.phi_w_hi_y;
    a.bcx_lo = h->d.bc_lo_x;
    a.bcx_hi = h->d.bc_hi_x;
    a.bcz_lo = h->d.bc_lo_z;
    a.bcz_hi = h->d.bc_hi_z;
    a.c = h->coef;
    a.status = h->status_dev;
    a.spin_limit = h->wait_limit;
    a.zwalk = h->zwalk;
    return a;
}

// Tensor maps for the TMA-staged steps, re-encoded when the velocity field changes.
static lbm_status ensure_tma_maps(lbm_cde_t h)
{
    const float* ua = h->ukind == LBM_U_FIELD ? h->ua : nullptr;
    if (h->tmaps_ok && h->tmaps_ua == ua) return LBM_OK;
    h->tmaps_ok = false;
    for (int b = 0; b < 2; ++b) {
        const bool ok = lbm::encode_tma_maps(h->state[b], h->phi[b], ua, (int)h->d.nx, (int)h->d.ny, &h->tmaps[b]);
        if (!ok) return fail(h, LBM_E_CUDA, "tensor map encoding failed (launch vec 7 / 8)");
    }
    h->tmaps_ok = true;
    h->tmaps_ua = ua;
    return LBM_OK;
}

// The status word latched by bounded device waits: LBM_E_TIMEOUT is reported
// (and the word cleared) by the next synchronising call.
static lbm_status check_status(lbm_cde_t h)
{
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (st != 0) {
        CK(h, cudaMemsetAsync(h->status_dev, 0, sizeof(int), h->st));
        return fail(h, (lbm_status)st, "a bounded wait in the TMA-staged step kernel timed out");
    }
    return LBM_OK;
}

static int ukind_internal(int k)
{
    return k == LBM_U_FIELD ? lbm::U_FIELD : (k == LBM_U_ROW_PROFILE ? lbm::U_ROW : lbm::U_NONE);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

lbm_status lbm_cde_desc_init(lbm_cde_desc* d, int32_t lattice, int64_t nx, int64_t ny, int64_t nz)
{
    if (!d) return fail(nullptr, LBM_E_ARG, "desc is NULL");
    std::memset(d, 0, sizeof(*d));
    d->lattice = lattice;
    d->storage = LBM_STORE_F32;
    d->nx = nx;
    d->ny = ny;
    d->nz = nz;
    d->bc_lo_y = d->bc_hi_y = LBM_BC_PERIODIC;
    d->bc_lo_x = d->bc_hi_x = d->bc_lo_z = d->bc_hi_z = LBM_BC_PERIODIC;
    d->alpha1 = d->alpha2 = NAN;
    for (int k = 0; k < 15; ++k) d->s[k] = NAN;
    d->tie_q_rates = 1;
    return LBM_OK;
}

lbm_status lbm_cde_create(const lbm_cde_desc* desc, lbm_cde_t* out)
{
    if (!desc || !out) return fail(nullptr, LBM_E_ARG, "desc/out is NULL");
    *out = nullptr;
    const lbm_cde_desc& d = *desc;
    if (d.lattice != LBM_D2Q9 && d.lattice != LBM_D3Q15)
        return fail(nullptr, LBM_E_ARG, "lattice must be LBM_D2Q9 or LBM_D3Q15");
    if (d.storage < LBM_STORE_F32 || d.storage > LBM_STORE_BF16_NEQ)
        return fail(nullptr, LBM_E_ARG, "bad storage");
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || (d.lattice == LBM_D2Q9 && d.nz != 1))
        return fail(nullptr, LBM_E_ARG, "bad grid size (D2Q9 needs nz = 1)");
    if (d.nx > (1LL << 30) || d.ny > 65535 || d.nz > 65535)
        return fail(nullptr, LBM_E_ARG, "grid too large (nx <= 2^30, ny, nz <= 65535)");
    const long long ncell = d.nx * d.ny * d.nz;
    if (ncell > (1LL << 40)) return fail(nullptr, LBM_E_ARG, "grid too large");
    for (int side = 0; side < 2; ++side) {
        const int b = side ? d.bc_hi_y : d.bc_lo_y;
        if (b < LBM_BC_PERIODIC || b > LBM_BC_DIRICHLET) return fail(nullptr, LBM_E_ARG, "bad bc");
    }
    if ((d.bc_lo_y == LBM_BC_PERIODIC) != (d.bc_hi_y == LBM_BC_PERIODIC))
        return fail(nullptr, LBM_E_ARG, "periodic y needs both y faces periodic");
    if (d.bc_lo_y != LBM_BC_PERIODIC && d.ny < 3)
        return fail(nullptr, LBM_E_ARG, "walls need ny >= 3");
    {
        const int fx[2] = {d.bc_lo_x, d.bc_hi_x}, fz[2] = {d.bc_lo_z, d.bc_hi_z};
        for (int k = 0; k < 2; ++k)
            if (fx[k] < LBM_BC_PERIODIC || fx[k] > LBM_BC_BOUNCEBACK || fz[k] < LBM_BC_PERIODIC ||
                fz[k] > LBM_BC_BOUNCEBACK)
                return fail(nullptr, LBM_E_ARG, "x and z faces take PERIODIC, NOFLUX_NODE or BOUNCEBACK");
        if ((fx[0] == LBM_BC_PERIODIC) != (fx[1] == LBM_BC_PERIODIC) ||
            (fz[0] == LBM_BC_PERIODIC) != (fz[1] == LBM_BC_PERIODIC))
            return fail(nullptr, LBM_E_ARG, "periodic x (z) needs both x (z) faces periodic");
        if (fx[0] != LBM_BC_PERIODIC && d.nx < 3) return fail(nullptr, LBM_E_ARG, "x walls need nx >= 3");
        if (fz[0] != LBM_BC_PERIODIC && (d.lattice != LBM_D3Q15 || d.nz < 3))
            return fail(nullptr, LBM_E_ARG, "z walls need D3Q15 and nz >= 3");
    }
    if ((d.alloc == nullptr) != (d.free_ == nullptr))
        return fail(nullptr, LBM_E_ARG, "alloc and free_ must both be set or both NULL");
    if (d.model < LBM_MRT_A || d.model > LBM_MRT_B3) return fail(nullptr, LBM_E_ARG, "bad model");
    if (d.model != LBM_MRT_A && d.lattice != LBM_D2Q9)
        return fail(nullptr, LBM_E_UNSUPPORTED, "the MRT-B models are D2Q9 only");
    if ((d.model == LBM_MRT_B1 || d.model == LBM_MRT_B2) &&
        (d.bc_lo_y == LBM_BC_DIRICHLET || d.bc_hi_y == LBM_BC_DIRICHLET))
        return fail(nullptr, LBM_E_UNSUPPORTED, "Dirichlet walls need an equilibrium linear in u (MRT-A, MRT-B3)");
    if ((d.model == LBM_MRT_B1 || d.model == LBM_MRT_B2) && d.storage != LBM_STORE_F32)
        return fail(nullptr, LBM_E_UNSUPPORTED, "MRT-B1/B2 need FP32 storage (their equilibria are not linear in u)");

    lbm_cde_t h = new (std::nothrow) lbm_cde_s();
    if (!h) return fail(nullptr, LBM_E_OOM, "host allocation failed");
    h->d = d;
    h->q = d.lattice;
    h->dim = d.lattice == LBM_D2Q9 ? 2 : 3;
    h->ncell = ncell;
    h->neq = d.storage != LBM_STORE_F32;
    h->elem = h->neq ? 2 : 4;
    h->st = static_cast<cudaStream_t>(d.stream);
    h->alpha1 = std::isnan(d.alpha1) ? (h->q == 9 ? -8.0 : -6.0 / 5.0) : d.alpha1;
    h->alpha2 = std::isnan(d.alpha2) ? (h->q == 9 ? 8.0 : 192.0) : d.alpha2;
    if (d.model != LBM_MRT_A) {
        // MRT-B1: m1 = (-2 + 3u^2), m2 = (1 - 3u^2) (Eq. 38); B2: m2 = (2 - 3u^2) (Eq. 39);
        // B3: Eq. 37. Their u = 0 parts are alpha1 = -8 and alpha2 = 4 (B1) or 8.
        h->alpha1 = -8.0;
        h->alpha2 = d.model == LBM_MRT_B1 ? 4.0 : 8.0;
    }
    const double defaults9[15] = {1.0, 1.1, 1.1, 0, 1.0, 0, 1.0, 1.2, 1.2, 0, 0, 0, 0, 0, 0};
    const double defaults15[15] = {1.0, 1.1, 1.1, 0, 1.0, 0, 1.0, 0, 1.0, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2};
    for (int k = 0; k < 15; ++k)
        h->s[k] = std::isnan(d.s[k]) ? (h->q == 9 ? defaults9[k] : defaults15[k]) : d.s[k];
    if (diffusion_factor(h->q, h->alpha1, h->alpha2, h->d.model) <= 0.0) {
        delete h;
        return fail(nullptr, LBM_E_ARG, "alpha1/alpha2 give a non-positive diffusion factor (Eq. 36 / A.6)");
    }
    for (int a = 0; a < h->dim; ++a) h->A[a * h->dim + a] = 1.0;  // replaced by set_D
    refresh_coef(h);

    const size_t plane_bytes = (size_t)ncell * h->elem;
    for (int b = 0; b < 2; ++b) {
        h->state[b] = dev_alloc(h, plane_bytes * h->q);
        if (!h->state[b]) {
            lbm_cde_destroy(h);
            return fail(nullptr, LBM_E_OOM, "state allocation failed");
        }
        if (h->neq) {
            h->phi[b] = static_cast<float*>(dev_alloc(h, (size_t)ncell * 4));
            if (!h->phi[b]) {
                lbm_cde_destroy(h);
                return fail(nullptr, LBM_E_OOM, "phi allocation failed");
            }
        }
    }
    long long nb = (ncell + 255) / 256;
    h->nparts = (int)(nb < 152 * 8 ? nb : 152 * 8);
    if (h->nparts < 1) h->nparts = 1;
    h->partials = static_cast<double*>(dev_alloc(h, sizeof(double) * (h->nparts + 1)));
    if (!h->partials) {
        lbm_cde_destroy(h);
        return fail(nullptr, LBM_E_OOM, "scratch allocation failed");
    }
    h->sum_dev = h->partials + h->nparts;
    h->status_dev = static_cast<int*>(dev_alloc(h, 16));
    if (!h->status_dev || cudaMemsetAsync(h->status_dev, 0, 16, h->st) != cudaSuccess) {
        lbm_cde_destroy(h);
        return fail(nullptr, LBM_E_OOM, "status word allocation failed");
    }
    {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            h->sms = n;
        cudaGetLastError();
    }
    // launch shape: 256 threads along x, cells per thread chosen for the row length
    h->cfg.block = d.nx >= 256 ? 256 : (d.nx >= 128 ? 128 : 64);
    h->cfg.vec = 1;
    *out = h;
    return LBM_OK;
}

lbm_status lbm_cde_destroy(lbm_cde_t h)
{
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->st);
    if (h->st_rec) cudaStreamSynchronize(h->st_rec);
    for (int b = 0; b < 2; ++b) {
        dev_free(h, h->state[b]);
        dev_free(h, h->phi[b]);
    }
    dev_free(h, h->phi_tmp);
    dev_free(h, h->partials);
    for (void* p : h->ck) dev_free(h, p);
    dev_free(h, h->seg);
    dev_free(h, h->seg2);
    for (int p = 0; p < 2; ++p) {
        if (h->ev_rec[p]) cudaEventDestroy(h->ev_rec[p]);
        if (h->ev_adj[p]) cudaEventDestroy(h->ev_adj[p]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->st_rec) cudaStreamDestroy(h->st_rec);
    dev_free(h, h->mu[0]);
    dev_free(h, h->mu[1]);
    dev_free(h, h->adj_partials);
    dev_free(h, h->phi0_saved);
    dev_free(h, h->status_dev);
    delete h;
    return LBM_OK;
}

lbm_status lbm_cde_set_D(lbm_cde_t h, const double* D)
{
    if (!h || !D) return fail(h, LBM_E_ARG, "NULL argument");
    const int n = h->dim;
    double scale = 0.0;
    for (int k = 0; k < n * n; ++k) {
        if (!std::isfinite(D[k])) return fail(h, LBM_E_NOT_SPD, "D has a non-finite entry");
        scale = std::fmax(scale, std::fabs(D[k]));
    }
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
            if (std::fabs(D[a * n + b] - D[b * n + a]) > 1e-12 * scale)
                return fail(h, LBM_E_NOT_SPD, "D is not symmetric");
    if (!spd(n, D)) return fail(h, LBM_E_NOT_SPD, "D is not positive definite");
    const double k = diffusion_factor(h->q, h->alpha1, h->alpha2, h->d.model);
    double Ainv[9], A[9];
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) Ainv[a * n + b] = D[a * n + b] / k + (a == b ? 0.5 : 0.0);
    if (!small_inverse(n, Ainv, A)) return fail(h, LBM_E_NOT_SPD, "A^-1 = D/k + I/2 is singular");
    for (int a = 0; a < n * n; ++a) h->A[a] = A[a];
    h->d_set = true;
    refresh_coef(h);
    return LBM_OK;
}

lbm_status lbm_cde_get_rates(lbm_cde_t h, double* A_out, double* s_out)
{
    if (!h || !A_out) return fail(h, LBM_E_ARG, "NULL argument");
    for (int a = 0; a < h->dim * h->dim; ++a) A_out[a] = h->A[a];
    if (s_out)
        for (int k = 0; k < 15; ++k) s_out[k] = h->coef.s[k];
    return LBM_OK;
}

lbm_status lbm_cde_set_velocity(lbm_cde_t h, int32_t kind, const float* a_dev, const float* sched_dev,
                                int64_t sched_len)
{
    if (!h) return fail(h, LBM_E_ARG, "NULL handle");
    if (kind != LBM_U_NONE && kind != LBM_U_FIELD && kind != LBM_U_ROW_PROFILE)
        return fail(h, LBM_E_ARG, "bad velocity kind");
    if (kind != LBM_U_NONE && !a_dev) return fail(h, LBM_E_ARG, "velocity pointer is NULL");
    if (sched_dev && (sched_len <= 0 || sched_len > (1LL << 26)))
        return fail(h, LBM_E_ARG, "sched_len must be in [1, 2^26]");
    h->ukind = kind;
    h->ua = kind == LBM_U_NONE ? nullptr : a_dev;
    h->sched = sched_dev;
    h->sched_len = sched_dev ? sched_len : 0;
    return LBM_OK;
}

lbm_status lbm_cde_set_phi(lbm_cde_t h, const float* phi_dev)
{
    if (!h || !phi_dev) return fail(h, LBM_E_ARG, "NULL argument");
    if (!h->d_set) return fail(h, LBM_E_STATE, "set_D must come before set_phi");
    h->cur = 0;
    h->t = 0;
    StepArgs a = make_args(h, 1);  // dst = state[0]
    a.dst = h->state[0];
    a.phi_dst = h->phi[0];
    CK(h, lbm::launch_init(h->q, h->d.storage, ukind_internal(h->ukind), phi_dev, a, h->st));
    h->ready = true;
    return LBM_OK;
}

lbm_status lbm_cde_step(lbm_cde_t h, int64_t nsteps)
{
    if (!h || nsteps < 0) return fail(h, LBM_E_ARG, "bad argument");
    if (!h->ready) return fail(h, LBM_E_STATE, "set_phi must come before step");
    const bool walls = h->d.bc_lo_y != LBM_BC_PERIODIC;
    const int uk = ukind_internal(h->ukind);
    const bool tma = (h->cfg.vec == 7 || h->cfg.vec == 8) && h->neq && h->q == 9;
    if (tma) {
        const lbm_status ts = ensure_tma_maps(h);
        if (ts != LBM_OK) return ts;
    }
    for (int64_t n = 0; n < nsteps; ++n) {
        StepArgs a = make_args(h, h->cur);
        if (tma) a.tma = &h->tmaps[h->cur];
        CK(h, lbm::launch_step(h->q, h->d.storage, uk, walls, h->cfg, a, h->st));
        h->cur ^= 1;
        h->t += 1;
    }
    return LBM_OK;
}

lbm_status lbm_cde_set_wait_limit(lbm_cde_t h, int64_t cycles)
{
    if (!h || cycles < 0) return fail(h, LBM_E_ARG, "bad argument");
    h->wait_limit = cycles;
    return LBM_OK;
}

lbm_status lbm_cde_set_zwalk(lbm_cde_t h, int32_t planes)
{
    if (!h || planes < 0) return fail(h, LBM_E_ARG, "bad argument");
    h->zwalk = planes;
    return LBM_OK;
}

lbm_status lbm_cde_set_launch(lbm_cde_t h, int32_t block, int32_t vec)
{
    if (!h) return fail(h, LBM_E_ARG, "NULL handle");
    const bool pair_ok = h->neq && h->d.nx % 2 == 0 && (long long)(h->q + 3) * h->ncell < (1LL << 31);
    const bool quad = h->q == 9 && h->d.nx % 4 == 0 && 12LL * h->ncell < (1LL << 31);
    const bool tma = h->neq && h->q == 9 && h->d.nx % 256 == 0 && 12LL * h->ncell < (1LL << 31);
    if (vec == 9) {
        if ((block != 256 && block != 128) || !h->neq || h->q != 15 || h->d.nx % 64 != 0 ||
            h->d.ny % (block / 32) != 0 || 18LL * h->ncell >= (1LL << 31))
            return fail(h, LBM_E_ARG, "vec 9 (D3Q15 z-walk 16-bit kernel) needs block 256 or 128, nx % 64 == 0, "
                                      "ny a multiple of block / 32 and 18 ncell < 2^31");
        h->cfg.block = block;
        h->cfg.vec = vec;
        return LBM_OK;
    }
    if (vec == 7 || vec == 8) {
        if (block != 128 || !tma)
            return fail(h, LBM_E_ARG, "vec 7 / 8 (TMA-staged D2Q9 16-bit kernel) needs block 128, "
                                      "nx % 256 == 0 and 12 ncell < 2^31");
        h->cfg.block = block;
        h->cfg.vec = vec;
        return LBM_OK;
    }
    if (block < 32 || block > 256 || block % 32 != 0 || vec < 1 || vec > 6 || vec == 3 || vec == 4 ||
        (vec == 5 && !pair_ok) || (vec == 6 && !quad))
        return fail(h, LBM_E_ARG, "block must be a multiple of 32 in [32, 256]; vec 1 or 2 (one or two nodes "
                                  "per thread), 5 (node-pair kernel, nx even, 16-bit storage) or 6 (D2Q9 "
                                  "node-quad kernel, nx % 4 == 0); vec 5 and 6 use 32-bit offsets: "
                                  "(q + 3) ncell < 2^31");
    h->cfg.block = block;
    h->cfg.vec = vec;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times the candidate launch shapes on the current state and keeps
// the fastest. Choices are cached in a text file (one "key block vec" line per
// configuration) named by LBMCDE_TUNE_CACHE, keyed by lattice, storage, grid,
// velocity kind, walls and GPU name.
// ---------------------------------------------------------------------------
static std::string tune_key(lbm_cde_t h)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string gpu(prop.name);
    for (char& ch : gpu)
        if (ch == ' ') ch = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "q%d_s%d_%lldx%lldx%lld_u%d_bc%d%d%d%d%d%d_%s", h->q, h->d.storage,
             (long long)h->d.nx, (long long)h->d.ny, (long long)h->d.nz, h->ukind, h->d.bc_lo_y, h->d.bc_hi_y,
             h->d.bc_lo_x, h->d.bc_hi_x, h->d.bc_lo_z, h->d.bc_hi_z, gpu.c_str());
    return buf;
}

static bool tune_cache_lookup(const std::string& key, int* block, int* vec)
{
    const char* path = getenv("LBMCDE_TUNE_CACHE");
    if (!path) return false;
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char k[256];
    int b = 0, v = 0;
    bool found = false;
    while (fscanf(fp, "%255s %d %d", k, &b, &v) == 3)
        if (key == k) {
            *block = b;
            *vec = v;
            found = true;
        }
    fclose(fp);
    return found;
}

static void tune_cache_store(const std::string& key, int block, int vec)
{
    const char* path = getenv("LBMCDE_TUNE_CACHE");
    if (!path) return;
    FILE* fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d\n", key.c_str(), block, vec);
    fclose(fp);
}

lbm_status lbm_cde_autotune(lbm_cde_t h, int64_t steps, int32_t* block_out, int32_t* vec_out)
{
    if (!h || steps < 1) return fail(h, LBM_E_ARG, "bad argument");
    if (!h->ready) return fail(h, LBM_E_STATE, "set_phi must come before autotune");
    const std::string key = tune_key(h);
    int cb = 0, cv = 0;
    if (tune_cache_lookup(key, &cb, &cv) && lbm_cde_set_launch(h, cb, cv) == LBM_OK) {
        if (block_out) *block_out = cb;
        if (vec_out) *vec_out = cv;
        return LBM_OK;
    }
    size_t sb = 0;
    lbm_cde_state_bytes(h, &sb);
    void* save = dev_alloc(h, sb);
    if (!save) return fail(h, LBM_E_OOM, "autotune buffer allocation failed");
    int64_t t0 = 0;
    lbm_status s = lbm_cde_get_state(h, save, &t0);
    if (s != LBM_OK) {
        dev_free(h, save);
        return s;
    }
    const LaunchCfg keep = h->cfg;
    float best = 1e30f;
    LaunchCfg best_cfg = keep;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // candidates: generic kernel (1 or 2 nodes per thread) at 64/128/256 threads;
    // for D2Q9 16-bit storage also the node-pair kernel at 64/128/256 threads; for
    // D3Q15 16-bit storage the node-pair kernel at 64 .. 256 threads; the node-quad
    // kernel (D2Q9), the TMA-staged D2Q9 kernel (16-bit storage) and the D3Q15
    // z-walk kernel where they apply
    std::vector<LaunchCfg> cand;
    for (int vec = 1; vec <= 2; ++vec)
        for (int b : {64, 128, 256}) cand.push_back(LaunchCfg{b, vec});
    if (h->q == 9 && h->neq && h->d.nx % 2 == 0 && 12LL * h->ncell < (1LL << 31))
        for (int b : {64, 128, 256}) cand.push_back(LaunchCfg{b, 5});
    if (h->q == 15 && h->neq && h->d.nx % 2 == 0 && 18LL * h->ncell < (1LL << 31))
        for (int b : {64, 96, 128, 192, 256}) cand.push_back(LaunchCfg{b, 5});
    if (h->q == 9 && h->d.nx % 4 == 0 && 12LL * h->ncell < (1LL << 31))
        for (int b : {64, 128, 256}) cand.push_back(LaunchCfg{b, 6});
    if (h->q == 15 && h->neq && h->d.nx % 64 == 0 && 18LL * h->ncell < (1LL << 31))
        for (int b : {128, 256})
            if (h->d.ny % (b / 32) == 0) cand.push_back(LaunchCfg{b, 9});
    if (h->neq && h->q == 9 && h->d.nx % 256 == 0 && 12LL * h->ncell < (1LL << 31) &&
        ensure_tma_maps(h) == LBM_OK) {   // tensor maps available
        cand.push_back(LaunchCfg{128, 7});
        cand.push_back(LaunchCfg{128, 8});
    }
    for (size_t ci = 0; ci < cand.size() && s == LBM_OK; ++ci) {
        h->cfg = cand[ci];
        s = lbm_cde_set_state(h, save, t0);
        if (s == LBM_OK) s = lbm_cde_step(h, 2);     // warm
        cudaEventRecord(e0, h->st);
        if (s == LBM_OK) s = lbm_cde_step(h, steps);
        cudaEventRecord(e1, h->st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (s == LBM_OK && ms < best) {
            best = ms;
            best_cfg = h->cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg = s == LBM_OK ? best_cfg : keep;
    lbm_status r = lbm_cde_set_state(h, save, t0);
    dev_free(h, save);
    if (s != LBM_OK) return s;
    if (r != LBM_OK) return r;
    tune_cache_store(key, h->cfg.block, h->cfg.vec);
    if (block_out) *block_out = h->cfg.block;
    if (vec_out) *vec_out = h->cfg.vec;
    return LBM_OK;
}

lbm_status lbm_cde_get_time(lbm_cde_t h, int64_t* t_out)
{
    if (!h || !t_out) return fail(h, LBM_E_ARG, "NULL argument");
    *t_out = h->t;
    return LBM_OK;
}

lbm_status lbm_cde_get_phi(lbm_cde_t h, float* phi_dev)
{
    if (!h || !phi_dev) return fail(h, LBM_E_ARG, "NULL argument");
    if (!h->ready) return fail(h, LBM_E_STATE, "no state yet");
    StepArgs a = make_args(h, h->cur);
    CK(h, lbm::launch_phi(h->q, h->d.storage, a, phi_dev, h->st));
    return LBM_OK;
}

lbm_status lbm_cde_sum_phi(lbm_cde_t h, double* out_host)
{
    if (!h || !out_host) return fail(h, LBM_E_ARG, "NULL argument");
    if (!h->ready) return fail(h, LBM_E_STATE, "no state yet");
    StepArgs a = make_args(h, h->cur);
    CK(h, lbm::launch_sum(h->q, h->d.storage, a, h->partials, h->nparts, h->sum_dev, h->st));
    CK(h, cudaMemcpyAsync(out_host, h->sum_dev, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    const lbm_status ds = check_status(h);   // synchronises
    if (ds != LBM_OK) return ds;
    if (!std::isfinite(*out_host)) return fail(h, LBM_E_NONFINITE, "sum of phi is not finite");
    return LBM_OK;
}

lbm_status lbm_cde_sync(lbm_cde_t h)
{
    if (!h) return fail(h, LBM_E_ARG, "NULL handle");
    return check_status(h);
}

lbm_status lbm_cde_state_bytes(lbm_cde_t h, size_t* bytes_out)
{
    if (!h || !bytes_out) return fail(h, LBM_E_ARG, "NULL argument");
    *bytes_out = (size_t)h->ncell * h->elem * h->q + (h->neq ? (size_t)h->ncell * 4 : 0);
    return LBM_OK;
}

lbm_status lbm_cde_get_state(lbm_cde_t h, void* dst, int64_t* t_out)
{
    if (!h || !dst) return fail(h, LBM_E_ARG, "NULL argument");
    if (!h->ready) return fail(h, LBM_E_STATE, "no state yet");
    const size_t fb = (size_t)h->ncell * h->elem * h->q;
    CK(h, cudaMemcpyAsync(dst, h->state[h->cur], fb, cudaMemcpyDefault, h->st));
    if (h->neq)
        CK(h, cudaMemcpyAsync(static_cast<char*>(dst) + fb, h->phi[h->cur], (size_t)h->ncell * 4,
                              cudaMemcpyDefault, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (t_out) *t_out = h->t;
    return LBM_OK;
}

lbm_status lbm_cde_set_state(lbm_cde_t h, const void* src, int64_t t)
{
    if (!h || !src || t < 0) return fail(h, LBM_E_ARG, "bad argument");
    const size_t fb = (size_t)h->ncell * h->elem * h->q;
    h->cur = 0;
    CK(h, cudaMemcpyAsync(h->state[0], src, fb, cudaMemcpyDefault, h->st));
    if (h->neq)
        CK(h, cudaMemcpyAsync(h->phi[0], static_cast<const char*>(src) + fb, (size_t)h->ncell * 4,
                              cudaMemcpyDefault, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    h->t = t;
    h->ready = true;
    return LBM_OK;
}

lbm_status lbm_cde_run_host(lbm_cde_t h, const float* phi0_host, int64_t nsteps, float* phi_out_host)
{
    if (!h || !phi0_host || !phi_out_host || nsteps < 0) return fail(h, LBM_E_ARG, "bad argument");
    if (!h->phi_tmp) {
        h->phi_tmp = static_cast<float*>(dev_alloc(h, (size_t)h->ncell * 4));
        if (!h->phi_tmp) return fail(h, LBM_E_OOM, "phi buffer allocation failed");
    }
    const size_t bytes = (size_t)h->ncell * 4;
    CK(h, cudaMemcpyAsync(h->phi_tmp, phi0_host, bytes, cudaMemcpyHostToDevice, h->st));
    lbm_status s = lbm_cde_set_phi(h, h->phi_tmp);
    if (s != LBM_OK) return s;
    s = lbm_cde_step(h, nsteps);
    if (s != LBM_OK) return s;
    s = lbm_cde_get_phi(h, h->phi_tmp);
    if (s != LBM_OK) return s;
    CK(h, cudaMemcpyAsync(phi_out_host, h->phi_tmp, bytes, cudaMemcpyDeviceToHost, h->st));
    return check_status(h);   // synchronises; reports a bounded wait that gave up
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------
int32_t lbm_cde_adjoint_ngrad(int32_t lattice) { return lbm::adjoint_ngrad(lattice == LBM_D3Q15 ? 15 : 9); }

static lbm_status adjoint_supported(lbm_cde_t h)
{
    if (h->d.storage != LBM_STORE_F32)
        return fail(h, LBM_E_UNSUPPORTED, "the adjoint needs FP32 state storage");
    if (!h->d_set) return fail(h, LBM_E_STATE, "set_D must come first");
    return LBM_OK;
}

// wall mode of the adjoint kernel: 0 periodic, 1 walls on the y faces only, 2 walls on x or z faces
static int adjoint_wmode(lbm_cde_t h)
{
    if (h->d.bc_lo_x != LBM_BC_PERIODIC || h->d.bc_lo_z != LBM_BC_PERIODIC) return 2;
    return h->d.bc_lo_y != LBM_BC_PERIODIC ? 1 : 0;
}

static lbm_status ensure_adjoint_buffers(lbm_cde_t h)
{
    const size_t sb = (size_t)h->ncell * 4 * h->q;
    for (int b = 0; b < 2; ++b)
        if (!h->mu[b]) {
            h->mu[b] = static_cast<float*>(dev_alloc(h, sb));
            if (!h->mu[b]) return fail(h, LBM_E_OOM, "adjoint state allocation failed");
        }
    if (!h->adj_partials) {
        const long long np = lbm::adjoint_partials_size(h->q, h->d.nx, h->d.ny, h->d.nz, h->sms);
        const int ng = lbm::adjoint_ngrad(h->q);
        h->adj_partials = static_cast<float*>(dev_alloc(h, sizeof(float) * (np + 2 * ng)));
        if (!h->adj_partials) return fail(h, LBM_E_OOM, "adjoint scratch allocation failed");
        h->grad_acc = reinterpret_cast<float2*>(h->adj_partials + np);   // np is even
    }
    return LBM_OK;
}

static lbm::AdjArgs make_adj(lbm_cde_t h, int64_t k, const float* mu_in, float* mu_out, const float* fprev,
                             float* du, float2* grad_acc)
{
    lbm::AdjArgs a{};
    a.mu_in = mu_in;
    a.mu_out = mu_out;
    a.fprev = fprev;
    a.ua = h->ua;
    a.sched = h->sched;
    a.sched_len = h->sched_len;
    a.k = k;
    a.srow = lbm::sched_row(k, h->sched ? h->sched_len : 0);
    a.srow_prev = lbm::sched_row(k - 1, h->sched ? h->sched_len : 0);
    a.phiw_lo = (float)h->d.phi_w_lo_y;
    a.phiw_hi = (float)h->d.phi_w_hi_y;
    a.rows = lbm::adjoint_rows(h->d.nx, h->d.ny, h->d.nz, h->sms);
    a.nx = (int)h->d.nx;
    a.ny = (int)h->d.ny;
    a.nz = (int)h->d.nz;
    a.ncell = h->ncell;
    a.bc_lo = h->d.bc_lo_y;
    a.bc_hi = h->d.bc_hi_y;
    a.bcx_lo = h->d.bc_lo_x;
    a.bcx_hi = h->d.bc_hi_x;
    a.bcz_lo = h->d.bc_lo_z;
    a.bcz_hi = h->d.bc_hi_z;
    a.c = h->coef;
    a.du_acc = du;
    a.partials = h->adj_partials;
    a.grad_acc = grad_acc;
    return a;
}

lbm_status lbm_cde_adjoint_step(lbm_cde_t h, int64_t k, const float* mu_k_dev, float* mu_prev_dev,
                                const float* f_prev_dev, float* grad_acc_dev, float* dL_da_dev)
{
    if (!h || !mu_k_dev || !mu_prev_dev || !f_prev_dev || !grad_acc_dev || k < 1)
        return fail(h, LBM_E_ARG, "bad argument");
    if (mu_k_dev == mu_prev_dev) return fail(h, LBM_E_ARG, "mu_k and mu_prev must not alias");
    lbm_status s = adjoint_supported(h);
    if (s != LBM_OK) return s;
    if (dL_da_dev && h->ukind != LBM_U_FIELD)
        return fail(h, LBM_E_UNSUPPORTED, "velocity gradients need a velocity field (LBM_U_FIELD)");
    if (dL_da_dev && (h->d.bc_lo_y == LBM_BC_DIRICHLET || h->d.bc_hi_y == LBM_BC_DIRICHLET))
        return fail(h, LBM_E_UNSUPPORTED, "velocity gradients are not formed with Dirichlet walls");
    s = ensure_adjoint_buffers(h);
    if (s != LBM_OK) return s;
    if (reinterpret_cast<uintptr_t>(grad_acc_dev) % 8 != 0) return fail(h, LBM_E_ARG, "grad_acc_dev not 8-byte aligned");
    lbm::AdjArgs a = make_adj(h, k, mu_k_dev, mu_prev_dev, f_prev_dev, dL_da_dev,
                              reinterpret_cast<float2*>(grad_acc_dev));
    CK(h, lbm::launch_adjoint(h->q, ukind_internal(h->ukind), adjoint_wmode(h), a, h->st, true));
    return LBM_OK;
}

lbm_status lbm_cde_grad_rates(lbm_cde_t h, const double* g, double* dL_dD_host, double* dL_ds_host)
{
    if (!h || !g) return fail(h, LBM_E_ARG, "NULL argument");
    const int n = h->dim, q = h->q;
    const double* GA = g;
    const double* GAC = g + n * n;
    const double* Gd = g + 2 * n * n;
    double s[15];
    for (int k = 0; k < 15; ++k) s[k] = h->coef.s[k];
    double dA[9] = {0}, ds[15] = {0};
    // S entries (Eq. 30-31 / A.5): A_ab, C_ab = (A_ab/2 - delta_ab) s_{q_b}, diagonal s_k.
    // The MRT-B models keep the unmodified S of Eq. 24 (C = 0): no coupling term.
    const bool coupled = h->d.model == LBM_MRT_A;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const double sq = s[4 + 2 * b];
            dA[a * n + b] = GA[a * n + b] + (coupled ? GAC[a * n + b] * sq / 2.0 : 0.0);
            if (coupled) ds[4 + 2 * b] += GAC[a * n + b] * (h->A[a * n + b] / 2.0 - (a == b ? 1.0 : 0.0));
        }
    for (int k = 1; k < q; ++k) {
        const bool flux = (k == 3 || k == 5 || (n == 3 && k == 7));
        if (!flux) ds[k] += Gd[k];
    }
    if (dL_ds_host)
        for (int k = 0; k < 15; ++k) dL_ds_host[k] = k < q ? ds[k] : 0.0;
    if (dL_dD_host) {
        // tied q-rates s_{q_b} = A_bb are functions of D as well
        if (h->d.tie_q_rates)
            for (int b = 0; b < n; ++b) dA[b * n + b] += ds[4 + 2 * b];
        // A = (D/k + I/2)^-1  =>  dL/dD = -(1/k) A^T dL/dA A^T
        const double kf = diffusion_factor(q, h->alpha1, h->alpha2, h->d.model);
        double T[9] = {0};
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int l = 0; l < n; ++l) acc += h->A[l * n + i] * dA[l * n + j];   // (A^T dA)_ij
                T[i * n + j] = acc;
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int l = 0; l < n; ++l) acc += T[i * n + l] * h->A[j * n + l];      // (T A^T)_ij
                dL_dD_host[i * n + j] = -acc / kf;
            }
    }
    return LBM_OK;
}

lbm_status lbm_cde_forward_ckpt(lbm_cde_t h, const float* phi0_dev, int64_t nsteps, int64_t every,
                                float* phiN_dev)
{
    if (!h || !phi0_dev || nsteps < 1 || every < 0) return fail(h, LBM_E_ARG, "bad argument");
    lbm_status s = adjoint_supported(h);
    if (s != LBM_OK) return s;
    if (every == 0) {
        every = (int64_t)std::ceil(std::sqrt((double)nsteps));
        if (every < 1) every = 1;
    }
    const int64_t nck = (nsteps + every - 1) / every;
    const size_t sb = (size_t)h->ncell * 4 * h->q;
    if ((int64_t)h->ck.size() != nck) {
        for (void* p : h->ck) dev_free(h, p);
        h->ck.assign(nck, nullptr);
        for (int64_t j = 0; j < nck; ++j) {
            h->ck[j] = dev_alloc(h, sb);
            if (!h->ck[j]) return fail(h, LBM_E_OOM, "checkpoint allocation failed");
        }
    }
    const int64_t segn = every > 1 ? every - 1 : 1;
    if (h->seg_states != segn) {
        dev_free(h, h->seg);
        dev_free(h, h->seg2);
        h->seg = dev_alloc(h, sb * segn);
        if (!h->seg) return fail(h, LBM_E_OOM, "segment allocation failed");
        // a second segment buffer lets the reverse sweep recompute the next
        // segment while it runs the adjoint steps of this one; without it the
        // sweep runs the two one after the other
        h->seg2 = nck > 1 ? dev_alloc(h, sb * segn) : nullptr;
        h->seg_states = segn;
    }
    if (!h->phi0_saved) {
        h->phi0_saved = static_cast<float*>(dev_alloc(h, (size_t)h->ncell * 4));
        if (!h->phi0_saved) return fail(h, LBM_E_OOM, "allocation failed");
    }
    CK(h, cudaMemcpyAsync(h->phi0_saved, phi0_dev, (size_t)h->ncell * 4, cudaMemcpyDeviceToDevice, h->st));
    s = lbm_cde_set_phi(h, phi0_dev);
    if (s != LBM_OK) return s;
    CK(h, cudaMemcpyAsync(h->ck[0], h->state[h->cur], sb, cudaMemcpyDeviceToDevice, h->st));
    for (int64_t k = 1; k <= nsteps; ++k) {
        s = lbm_cde_step(h, 1);
        if (s != LBM_OK) return s;
        if (k % every == 0 && k < nsteps)
            CK(h, cudaMemcpyAsync(h->ck[k / every], h->state[h->cur], sb, cudaMemcpyDeviceToDevice, h->st));
    }
    if (phiN_dev) {
        s = lbm_cde_get_phi(h, phiN_dev);
        if (s != LBM_OK) return s;
    }
    h->ck_every = every;
    h->ck_nsteps = nsteps;
    h->have_fwd = true;
    return LBM_OK;
}

lbm_status lbm_cde_backward(lbm_cde_t h, const float* dL_dphiN_dev, float* dL_dphi0_dev, double* dL_dD_host,
                            double* dL_ds_host, float* dL_da_dev)
{
    if (!h || !dL_dphiN_dev || !dL_dphi0_dev) return fail(h, LBM_E_ARG, "NULL argument");
    if (!h->have_fwd) return fail(h, LBM_E_STATE, "lbm_cde_forward_ckpt must come first");
    lbm_status s = adjoint_supported(h);
    if (s != LBM_OK) return s;
    if (dL_da_dev && h->ukind != LBM_U_FIELD)
        return fail(h, LBM_E_UNSUPPORTED, "velocity gradients need a velocity field (LBM_U_FIELD)");
    if (dL_da_dev && (h->d.bc_lo_y == LBM_BC_DIRICHLET || h->d.bc_hi_y == LBM_BC_DIRICHLET))
        return fail(h, LBM_E_UNSUPPORTED, "velocity gradients are not formed with Dirichlet walls");
    s = ensure_adjoint_buffers(h);
    if (s != LBM_OK) return s;
    const int ng = lbm::adjoint_ngrad(h->q);
    const size_t sb = (size_t)h->ncell * 4 * h->q;
    const int uk = ukind_internal(h->ukind);
    const bool walls = h->d.bc_lo_y != LBM_BC_PERIODIC;
    // optional per-phase timing: one event before and after each segment's recompute
    // and after its reverse steps (lbm_cde_set_profiling)
    struct Events {
        std::vector<cudaEvent_t> e;
        std::vector<int> kind;   // 0: recompute boundary, 1: reverse-step boundary, 2: sweep
        ~Events() { for (cudaEvent_t x : e) cudaEventDestroy(x); }
        cudaError_t mark(cudaStream_t st, int k = 2)
        {
            cudaEvent_t x = nullptr;
            cudaError_t r = cudaEventCreate(&x);
            if (r != cudaSuccess) return r;
            e.push_back(x);
            kind.push_back(k);
            return cudaEventRecord(x, st);
        }
    } ev;
    if (h->prof) CK(h, ev.mark(h->st));
    CK(h, cudaMemsetAsync(h->grad_acc, 0, sizeof(float2) * ng, h->st));
    const long long slice = lbm::adjoint_slice_size(h->q, h->d.nx, h->d.ny, h->d.nz, h->sms);
    int nslice = 0;   // reverse steps since the last gradient reduction
    if (dL_da_dev) CK(h, cudaMemsetAsync(dL_da_dev, 0, (size_t)h->ncell * 4 * h->dim, h->st));
    CK(h, lbm::launch_adjoint_seed(dL_dphiN_dev, h->mu[0], h->ncell, h->q, h->st));
    int cur = 0;
    const int64_t K = h->ck_every, Nst = h->ck_nsteps;
    const int64_t nck = (int64_t)h->ck.size();
    // Overlapped sweep (two segment buffers): segment j's states sit in buffer
    // j & 1; the recompute of segment j - 1 runs on st_rec while the adjoint steps
    // of segment j run on the handle's stream, ordered by events (a buffer is
    // refilled only after the adjoint steps that read it). Otherwise the
    // recompute and the adjoint steps of each segment run in turn.
    bool overlap = h->seg2 != nullptr;
    if (overlap && !h->st_rec) {
        if (cudaStreamCreateWithFlags(&h->st_rec, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            h->st_rec = nullptr;
        } else {
            bool ok = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming) == cudaSuccess;
            for (int p = 0; p < 2 && ok; ++p)
                ok = cudaEventCreateWithFlags(&h->ev_rec[p], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&h->ev_adj[p], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) return fail(h, LBM_E_CUDA, "event creation failed");
        }
    }
    overlap = overlap && h->st_rec != nullptr;
    void* segbuf[2] = {h->seg, overlap ? h->seg2 : h->seg};
    auto seg_state = [&](int64_t j, int64_t t) -> float* {   // B_{jK + t}
        if (t == 0) return static_cast<float*>(h->ck[j]);
        return reinterpret_cast<float*>(static_cast<char*>(segbuf[j & 1]) + sb * (t - 1));
    };
    // recompute B_{jK+1} .. B_{end-1} of segment j from its checkpoint, on stream rs
    auto recompute = [&](int64_t j, cudaStream_t rs) -> lbm_status {
        const int64_t start = j * K, end = std::min(start + K, Nst);
        for (int64_t t = 1; t < end - start; ++t) {
            StepArgs a = make_args(h, 0);
            a.src = seg_state(j, t - 1);
            a.dst = seg_state(j, t);
            set_step(a, start + t);
            CK(h, lbm::launch_step(h->q, LBM_STORE_F32, uk, walls, h->cfg, a, rs));
        }
        return LBM_OK;
    };
    if (overlap) {
        CK(h, cudaEventRecord(h->ev_start, h->st));   // checkpoints and seed are ordered before
        CK(h, cudaStreamWaitEvent(h->st_rec, h->ev_start, 0));
        if (h->prof) CK(h, ev.mark(h->st_rec, 0));
        s = recompute(nck - 1, h->st_rec);
        if (s != LBM_OK) return s;
        if (h->prof) CK(h, ev.mark(h->st_rec, 0));
        CK(h, cudaEventRecord(h->ev_rec[(nck - 1) & 1], h->st_rec));
    }
    for (int64_t j = nck - 1; j >= 0; --j) {
        const int64_t start = j * K;
        const int64_t end = std::min(start + K, Nst);
        if (overlap) {
            CK(h, cudaStreamWaitEvent(h->st, h->ev_rec[j & 1], 0));
            if (j >= 1) {
                // buffer (j - 1) & 1 was last read by the adjoint steps of segment j + 1
                if (j + 1 < nck) CK(h, cudaStreamWaitEvent(h->st_rec, h->ev_adj[(j + 1) & 1], 0));
                if (h->prof) CK(h, ev.mark(h->st_rec, 0));
                s = recompute(j - 1, h->st_rec);
                if (s != LBM_OK) return s;
                if (h->prof) CK(h, ev.mark(h->st_rec, 0));
                CK(h, cudaEventRecord(h->ev_rec[(j - 1) & 1], h->st_rec));
            }
        } else {
            if (h->prof) CK(h, ev.mark(h->st, 0));
            s = recompute(j, h->st);
            if (s != LBM_OK) return s;
            if (h->prof) CK(h, ev.mark(h->st, 0));
        }
        if (h->prof) CK(h, ev.mark(h->st, 1));
        for (int64_t k = end; k > start; --k) {
            lbm::AdjArgs a = make_adj(h, k, h->mu[cur], h->mu[1 - cur], seg_state(j, k - 1 - start), dL_da_dev,
                                      h->grad_acc);
            a.partials = h->adj_partials + nslice * slice;
            CK(h, lbm::launch_adjoint(h->q, uk, adjoint_wmode(h), a, h->st, false));
            if (++nslice == lbm::ADJ_SLICES) {
                CK(h, lbm::launch_grad_reduce(h->q, a, h->adj_partials, nslice, slice, h->st));
                nslice = 0;
            }
            cur ^= 1;
        }
        if (h->prof) CK(h, ev.mark(h->st, 1));
        if (overlap) CK(h, cudaEventRecord(h->ev_adj[j & 1], h->st));
    }
    lbm::AdjArgs a0 = make_adj(h, 0, h->mu[cur], nullptr, nullptr, dL_da_dev, h->grad_acc);
    if (nslice > 0) CK(h, lbm::launch_grad_reduce(h->q, a0, h->adj_partials, nslice, slice, h->st));
    CK(h, lbm::launch_adjoint_init(h->q, uk, a0, h->phi0_saved, dL_dphi0_dev, h->st));
    float2 gc[33];
    CK(h, cudaMemcpyAsync(gc, h->grad_acc, sizeof(float2) * ng, cudaMemcpyDeviceToHost, h->st));
    if (h->prof) CK(h, ev.mark(h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (h->prof) {
        // events: the first and the last mark the whole sweep on the handle's
        // stream; in between, pairs (before, after) of one segment's recompute and
        // of one segment's reverse steps, in the order they were issued
        double rec = 0.0, adj = 0.0;
        float ms = 0.f;
        const size_t ne = ev.e.size();
        for (size_t j = 1; j + 2 < ne; j += 2) {
            CK(h, cudaEventElapsedTime(&ms, ev.e[j], ev.e[j + 1]));
            (ev.kind[j] ? adj : rec) += ms;
        }
        CK(h, cudaEventElapsedTime(&ms, ev.e[0], ev.e[ne - 1]));
        h->prof_ms[0] = rec;
        h->prof_ms[1] = adj;
        h->prof_ms[2] = ms;
    }
    double g[33];
    for (int j = 0; j < ng; ++j) g[j] = (double)gc[j].x + (double)gc[j].y;   // compensated sum, host FP64
    return lbm_cde_grad_rates(h, g, dL_dD_host, dL_ds_host);
}

lbm_status lbm_cde_set_profiling(lbm_cde_t h, int32_t on)
{
    if (!h) return fail(h, LBM_E_ARG, "NULL handle");
    h->prof = on != 0;
    return LBM_OK;
}

lbm_status lbm_cde_backward_phases(lbm_cde_t h, double* ms_out)
{
    if (!h || !ms_out) return fail(h, LBM_E_ARG, "NULL argument");
    for (int j = 0; j < 3; ++j) ms_out[j] = h->prof_ms[j];
    return LBM_OK;
}

const char* lbm_cde_last_error(lbm_cde_t h)
{
    return h ? h->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
