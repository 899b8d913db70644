// Internal declarations shared by the CUDA translation units of the solver.
// Not part of the public C ABI (include/lbm_cde.h).
#pragma once

#include <cuda.h>            // CUtensorMap (tensor maps of the TMA-staged step)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {

enum Store { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum UKind { U_NONE = 0, U_FIELD = 1, U_ROW = 2 };
enum Bc { BC_PERIODIC = 0, BC_NOFLUX = 1, BC_BOUNCE = 2, BC_DIRICHLET = 3 };

// Relaxation and equilibrium constants of one solver, passed by value to
// every kernel (they live in the kernel parameter bank, i.e. constant cache).
struct Coef {
    // m^eq per unit phi for the two scalar moments:
    //   D2Q9  (Eq. 15b-c): m1 = alpha1/4, m2 = alpha2/4
    //   D3Q15 (Eq. A.3b-c): m1 = 5 alpha1/6, m2 = alpha2/24
    float meq1, meq2;
    float s[15];   // diagonal rates (entries 3, 5, 7 unused)
    float A[9];    // flux block (row-major dim x dim)
    // Coupling of flux row a to q-moment column b (Eq. 30a-b, A.5):
    //   (A_ab / 2 - delta_ab) * s_{q-row of b}
    float C[9];
    // f^eq_i = phi * (w_i + k_i e_i.u), Eq. 17 / its D3Q15 counterpart
    float w0, wa, wd, ka, kd;
    // u^2 terms of the MRT-B1/B2 equilibria (Eq. 38-39), zero for MRT-A/B3:
    //   m1 += b1 |u|^2 phi, m2 += b2 |u|^2 phi, m7 = g7 (ux^2 - uy^2) phi, m8 = g8 ux uy phi
    float b1, b2, g7, g8;
    // Offset forms (linear equilibria): the relaxation and the 1/|M_k|^2
    // scaling folded together, a_k = (m' - m^eq)_k / |M_k|^2 from dl = m - m^eq:
    //   ro[k] = (1 - s_k) / |M_k|^2 for the diagonal rows;
    //   D2Q9: fr[4 r + j], flux row 3 + 2 r on dl_3, dl_4, dl_5, dl_6
    //         ((delta_r0 - A_r0) / 6, -C_r0 / 6, (delta_r1 - A_r1) / 6, -C_r1 / 6);
    //   D3Q15: fr[6 r + 2 b + j], flux row 3 + 2 r on dl_{3 + 2 b} (j = 0) and
    //         dl_{4 + 2 b} (j = 1): (delta_rb - A_rb) / |M_3|^2, -C_rb / |M_3|^2
    float ro[15];
    float fr[18];
    // sum_i w_i - 1 with the FP32 weights the 16-bit decode adds back (w0 + 4 wa
    // + 4 wd for D2Q9, w0 + 6 wa + 8 wd for D3Q15): the rest offset g_0 carries
    // -phi eps0 so that decode and store conserve mass in FP32 as they do exactly
    float eps0;
};

// Fills ro and fr from s, A and C (D2Q9 or D3Q15; host side).
inline void fold_offset_coef(Coef& c, int q = 9)
{
    if (q == 9) {
        const double n2[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};
        for (int k = 0; k < 9; ++k) c.ro[k] = (float)((1.0 - (double)c.s[k]) / n2[k]);
        for (int r = 0; r < 2; ++r) {
            c.fr[4 * r + 0] = (float)(((r == 0 ? 1.0 : 0.0) - (double)c.A[2 * r + 0]) / 6.0);
            c.fr[4 * r + 1] = (float)(-(double)c.C[2 * r + 0] / 6.0);
            c.fr[4 * r + 2] = (float)(((r == 1 ? 1.0 : 0.0) - (double)c.A[2 * r + 1]) / 6.0);
            c.fr[4 * r + 3] = (float)(-(double)c.C[2 * r + 1] / 6.0);
        }
        return;
    }
    // D3Q15 row norms |M_k|^2 of Eq. A.2
    const double n2[15] = {15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8};
    for (int k = 0; k < 15; ++k) c.ro[k] = (float)((1.0 - (double)c.s[k]) / n2[k]);
    for (int r = 0; r < 3; ++r)
        for (int b = 0; b < 3; ++b) {
            c.fr[6 * r + 2 * b] = (float)(((r == b ? 1.0 : 0.0) - (double)c.A[3 * r + b]) / n2[3]);
            c.fr[6 * r + 2 * b + 1] = (float)(-(double)c.C[3 * r + b] / n2[3]);
        }
}

// Tensor maps of the TMA-staged D2Q9 step (k_step_tma_d2q9) for one source
// buffer: each pair is the 256-column box of one grid row and its halo box.
struct TmaMaps {
    CUtensorMap g, gh;    // 16-bit offsets [9][ny][nx]: boxes (256, 1, 9) and (8, 1, 9)
    CUtensorMap p, ph;    // phi [ny][nx]: boxes (256, 1) and (4, 1)
    CUtensorMap u, uh;    // velocity factors [2][ny][nx]: boxes (256, 1, 2) and (4, 1, 2)
};

struct StepArgs {
    const void* src;      // state planes [q][ncell] (float or 16-bit)
    void* dst;
    const float* phi_src; // phi planes of the 16-bit forms
    float* phi_dst;
    const float* ua;      // velocity a(x) (FIELD: [dim][ncell], ROW: [dim][ny])
    const float* sched;   // [sched_len][dim] or nullptr
    long long sched_len;
    long long k;          // this step computes f(k) and collides with u(k)
    int srow_now;         // schedule rows of u(k) and u(k-1): k mod sched_len,
    int srow_prev;        // (k-1) mod sched_len, or -1 without a schedule
    int nx, ny, nz;
    long long ncell;
    int bc_lo, bc_hi;     // y faces
    float phiw_lo, phiw_hi;
    int bcx_lo, bcx_hi;   // x faces (k_step_box only)
    int bcz_lo, bcz_hi;   // z faces (k_step_box only)
    Coef c;
    int* status;          // device status word (LBM_E_TIMEOUT from a bounded wait) or nullptr
    long long spin_limit; // SM clock cycles a bounded wait may take (0: give up at once)
    const TmaMaps* tma;   // host pointer: tensor maps of src / phi_src / ua, or nullptr
    int zwalk;            // D3Q15 z-walk kernel: planes per CTA (0: chosen by the launcher)
};

// One reverse-time step (lbm_adjoint.cu).
struct AdjArgs {
    const float* mu_in;   // adjoint of the post-collision state B_k [q][ncell]
    float* mu_out;        // adjoint of B_{k-1}
    const float* fprev;   // forward state B_{k-1} (FP32) [q][ncell]
    const float* ua;
    const float* sched;
    long long sched_len;
    long long k;          // the forward step being reversed (collision with u(k))
    int srow;             // k mod sched_len, or -1 without a schedule
    int srow_prev;        // (k - 1) mod sched_len, or -1: u(k - 1) of the Dirichlet fill
    float phiw_lo, phiw_hi;   // Dirichlet wall values (y faces)
    int rows;             // grid rows per block (adjoint_rows)
    int nx, ny, nz;
    long long ncell;
    int bc_lo, bc_hi;     // y faces
    int bcx_lo, bcx_hi;   // x faces (wall mode 2)
    int bcz_lo, bcz_hi;   // z faces (wall mode 2)
    Coef c;
    float* du_acc;        // dL/da accumulator [dim][ncell] (FIELD velocity) or nullptr
    float* partials;      // per-block gradient partials [ngrad][nblocks] (one slice per step)
    float2* grad_acc;     // [ngrad] running compensated sums (value = x + y): G_A[dim][dim],
                          // G_AC[dim][dim], G_diag[q]
};

// Row of a schedule of length len for step k (k mod len), -1 without one;
// computed on the host so that no kernel divides by the schedule length.
inline int sched_row(long long k, long long len)
{
    if (len <= 0) return -1;
    long long r = k % len;
    return (int)(r < 0 ? r + len : r);
}

inline void set_step(StepArgs& a, long long k)
{
    a.k = k;
    a.srow_now = sched_row(k, a.sched ? a.sched_len : 0);
    a.srow_prev = sched_row(k - 1, a.sched ? a.sched_len : 0);
}

// The node-quad D2Q9 kernel needs nx % 4 == 0, int offsets and a 16-byte
// aligned velocity field (it reads four nodes per vector load).
inline bool quad_ok(const StepArgs& a, int ukind)
{
    return a.nx % 4 == 0 && a.nz == 1 && 12LL * a.ncell < (1LL << 31) &&
           (ukind != U_FIELD || (reinterpret_cast<uintptr_t>(a.ua) & 15) == 0);
}

// The node-pair kernels need nx even, int offsets ((q + 3) ncell < 2^31) and
// an 8-byte aligned velocity field (they read two nodes per vector load).
inline bool pair_ok(const StepArgs& a, int ukind, int q)
{
    return a.nx % 2 == 0 && (long long)(q + 3) * a.ncell < (1LL << 31) &&
           (ukind != U_FIELD || (reinterpret_cast<uintptr_t>(a.ua) & 7) == 0);
}

// The TMA-staged D2Q9 kernel needs 256-column strips (nx % 256 == 0), int
// offsets, a 16-byte aligned velocity field and the tensor maps of the source.
inline bool tma_ok(const StepArgs& a, int ukind)
{
    return a.tma != nullptr && a.nx % 256 == 0 && a.nz == 1 && 12LL * a.ncell < (1LL << 31) &&
           (ukind != U_FIELD || (reinterpret_cast<uintptr_t>(a.ua) & 15) == 0);
}

// The D3Q15 z-walk kernel needs 64-column tiles (nx % 64 == 0), ty-row tiles
// (ny % ty == 0), int offsets and 16-byte aligned offsets, phi and velocity
// fields (its shared-memory fills are 16-byte copies).
inline bool zw_ok(const StepArgs& a, int ukind, int ty)
{
    return a.nx % 64 == 0 && a.ny % ty == 0 && 18LL * a.ncell < (1LL << 31) &&
           (reinterpret_cast<uintptr_t>(a.phi_src) & 15) == 0 && (reinterpret_cast<uintptr_t>(a.src) & 15) == 0 &&
           (ukind != U_FIELD || (reinterpret_cast<uintptr_t>(a.ua) & 15) == 0);
}

// Encode the tensor maps for one source buffer (lbm_tma.cu); false if the
// driver entry point is missing or the layout breaks a tensor-map rule.
bool encode_tma_maps(const void* g, const float* phi, const float* ua, int nx, int ny, TmaMaps* out);

struct LaunchCfg {
    int block;   // threads per block (multiple of 32)
    int vec;     // cells per thread along x (1, 2 or 4)
};

// Kernel launchers (lbm_kernels.cu). Each returns the cudaError_t of the launch.
cudaError_t launch_step(int q, int store, int ukind, bool walls, LaunchCfg cfg,
                        const StepArgs& a, cudaStream_t st);
cudaError_t launch_init(int q, int store, int ukind, const float* phi0, const StepArgs& a,
                        cudaStream_t st);
cudaError_t launch_phi(int q, int store, const StepArgs& a, float* phi_out, cudaStream_t st);
cudaError_t launch_sum(int q, int store, const StepArgs& a, double* partials, int nblocks,
                       double* out_dev, cudaStream_t st);

// reduce = true: also add the block partials to grad_acc (one step at a time);
// a backward sweep writes the partials of up to ADJ_SLICES consecutive steps to
// separate slices (AdjArgs::partials = base + slice * adjoint_slice_size) and
// reduces them together with launch_grad_reduce.
// wmode: 0 periodic, 1 walls on the y faces only, 2 walls on x or z faces (any face)
cudaError_t launch_adjoint(int q, int ukind, int wmode, const AdjArgs& a, cudaStream_t st, bool reduce);
cudaError_t launch_grad_reduce(int q, const AdjArgs& a, float* base, int nslice, long long slice, cudaStream_t st);
long long adjoint_slice_size(int q, long long nx, long long ny, long long nz, int sms);
constexpr int ADJ_SLICES = 16;   // reverse steps whose block partials are kept apart before one reduction
cudaError_t launch_adjoint_init(int q, int ukind, const AdjArgs& a, const float* phi0, float* dphi0,
                                cudaStream_t st);
cudaError_t launch_adjoint_seed(const float* g, float* mu, long long ncell, int q, cudaStream_t st);
long long adjoint_partials_size(int q, long long nx, long long ny, long long nz, int sms);   // in floats
int adjoint_rows(long long nx, long long ny, long long nz, int sms);
int adjoint_ngrad(int q);

}  // namespace lbm
