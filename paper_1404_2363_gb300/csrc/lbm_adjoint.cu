// Reverse-time (adjoint) step of the fused stream + collide kernel.
//
// For a fixed velocity field one step is linear in the distributions: with the
// stored post-collision state B_k = C_k P B_{k-1} (P = pull-stream and walls,
// C_k = M^-1 [I - S (I - v e_0^T)] M the collision with m^eq = phi v(u(k)),
// Eq. 11-15, 30-31), the adjoint mu_k = dL/dB_k obeys
//     mu_{k-1} = P^T C_k^T mu_k .
// One thread per node y: it applies C_k^T to mu_k(y) in moment space,
//     a = diag(1/|M_r|^2) M mu,   b = S^T a,   c = a - b + e_0 (v . b),   nu = M^T c,
// then pushes nu_i to mu_{k-1,i}(y - e_i) (the transpose of the forward pull,
// which read that same address), with the transposed wall rules. The forward
// pre-collision state f_k = P B_{k-1} is pulled again to form the parameter
// partials  dL/dS_rc = -sum a_r (m - m^eq)_c  and the velocity partials
//     dL/du_a = phi (b_{j_a} - b_{q_a})   (j_a, q_a: flux and energy-flux rows).
// Gradient partials are summed in FP32 per thread, warp and block, and over
// blocks and steps as compensated FP32 sums (error-free TwoSum: value = sum +
// compensation), in a fixed order; no FP64 arithmetic runs on the GPU here.
#include "lbm_device.cuh"

namespace lbm {

template <class L>
__host__ __device__ constexpr int ngrad() { return 2 * L::DIM * L::DIM + L::Q; }

// Error-free transformation of a + b (TwoSum, Knuth): returns fl(a + b) and
// sets e so that a + b = s + e exactly. Explicit roundings: never reassociated.
__device__ __forceinline__ float two_sum(float a, float b, float& e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// compensated sums (x: sum, y: accumulated rounding errors)
__device__ __forceinline__ void csum_add(float2& acc, float v)
{
    float e;
    acc.x = two_sum(acc.x, v, e);
    acc.y = __fadd_rn(acc.y, e);
}

__device__ __forceinline__ void csum_merge(float2& acc, float2 o)
{
    float e;
    acc.x = two_sum(acc.x, o.x, e);
    acc.y = __fadd_rn(__fadd_rn(acc.y, o.y), e);
}

// Rows handled by one block of the adjoint kernel (AdjArgs::rows): the gradient
// partials of that many nodes per thread are summed in registers before the
// block reduction. At most ADJ_ROWS; fewer on small grids, so that the grid
// still holds about three resident blocks per SM. (A grid of exactly one
// resident wave, each block walking rows gridDim.y apart, measured slower:
// 2.99x instead of 2.55x a forward step at 4096^2.)
constexpr int ADJ_ROWS = 8;

int adjoint_rows(long long nx, long long ny, long long nz, int sms)
{
    int rows = ADJ_ROWS;
    while (rows > 1 && ((nx + 255) / 256) * ((ny + rows - 1) / rows) * nz < (long long)sms * 3) rows /= 2;
    return rows;
}

// DA: the velocity-field gradient is accumulated (UK == U_FIELD only); its
// running values are requested with the other loads of the node, and the
// instance runs at 3 blocks per SM (80 registers) to hold them.
// IX: int when every plane offset fits in 31 bits (fewer address
// instructions), long long otherwise. The maps M f, M mu and M^T c use the
// same sums and differences of same-speed populations as the forward step
// (moments / populations): the kernel is bound by its instruction issue.
// WM: 0 periodic; 1 walls on the y faces (the rules in place below); 2 walls
// on any face (BOX): each pull source found as in k_step_box, and the push
// scatters nu_i to the address the forward pull of population i read: the
// regular source (j, x - e_j), or for a bounce-back face the node's own
// reversed population (opp j, x), j being i or, where the source lies beyond
// NOFLUX_NODE faces, i reflected in those axes. Each address is read by the
// pulls of one node only, so every thread writes its own addresses: (j, x - e_j)
// for the sources in range, and (k, x) for the populations that leave through
// a wall (zero unless a bounce-back pull read them).
// QUAD: the u^2 terms of the MRT-B1/B2 equilibria (D2Q9 with a velocity only);
// a compile-time choice: behind a run-time test the kernel executed 7 % more
// instructions for the other models, which never take them.
template <class L, int UK, int WM, bool DA, typename IX, bool QUAD>
__global__ void __launch_bounds__(256, (L::Q == 9 && !DA && WM < 2) ? 4 : 3) k_adjoint(const AdjArgs a)
{
    static_assert(!QUAD || (L::Q == 9 && UK != U_NONE), "u^2 terms only for D2Q9 with a velocity");
    constexpr bool WALLS = WM == 1, BOX = WM == 2;
    constexpr int Q = L::Q, DIM = L::DIM, NG = ngrad<L>();
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.z;
    const IX N = (IX)a.ncell;
    const bool live = x < nx;
    const int xc = live ? x : nx - 1;
    const int xs[3] = {xc + 1 == nx ? 0 : xc + 1, xc, xc == 0 ? nx - 1 : xc - 1};
    const int zs[3] = {z + 1 == nz ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};
    const Coef& c = a.c;
    float s_now[3];
    sched_row_at(a.sched, a.srow, DIM, s_now);

    float g[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) g[j] = 0.f;

    const int y0 = blockIdx.y * a.rows;
#pragma unroll 1
    for (int y = y0; y < y0 + a.rows && y < ny; ++y) {
        const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
        // row offsets of the source rows (y - e_y, z - e_z)
        IX roff[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                roff[b][d] = DIM == 2 ? (IX)nx * (IX)ys[b] : (IX)nx * ((IX)ys[b] + (IX)ny * (IX)zs[d]);
        const IX cell = (IX)xc + roff[1][1];
        // pull source of population i = push target of its adjoint
        auto tgt = [&](int i) -> IX { return (IX)xs[L::ex(i) + 1] + roff[L::ey(i) + 1][L::ez(i) + 1]; };
        float mu[Q], f[Q];
        float du_old[DIM];
        if (DA && live) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) du_old[d] = a.du_acc[(IX)d * N + cell];
        }
        // BOX: pull source of every population (in range after periodic wrap, or
        // beyond a wall: bounce-back flag, mask of the NOFLUX_NODE axes)
        IX bsrc[Q];
        bool bout[Q], bbb[Q];
        int bnf[Q];
        if constexpr (BOX) {
            const int pos[3] = {xc, y, z}, n3[3] = {nx, ny, nz};
            const int klo[3] = {a.bcx_lo, a.bc_lo, a.bcz_lo}, khi[3] = {a.bcx_hi, a.bc_hi, a.bcz_hi};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
                int sp[3];
                bout[i] = false;
                bbb[i] = false;
                bnf[i] = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    sp[d] = pos[d] - e[d];
                    if (e[d] == 0) continue;
                    if (klo[d] == BC_PERIODIC) {
                        sp[d] = sp[d] < 0 ? sp[d] + n3[d] : (sp[d] >= n3[d] ? sp[d] - n3[d] : sp[d]);
                    } else if (sp[d] < 0 || sp[d] >= n3[d]) {
                        const int kind = sp[d] < 0 ? klo[d] : khi[d];
                        bout[i] = true;
                        bbb[i] = bbb[i] || kind == BC_BOUNCE;
                        if (kind == BC_NOFLUX) bnf[i] |= 1 << d;
                    }
                }
                bsrc[i] = bout[i] ? cell : (IX)sp[0] + (IX)nx * ((IX)sp[1] + (IX)ny * (IX)sp[2]);
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            mu[i] = __ldg(a.mu_in + (IX)i * N + cell);
            if constexpr (BOX) {
                f[i] = !bout[i] ? __ldg(a.fprev + (IX)i * N + bsrc[i])
                                : (bbb[i] ? __ldg(a.fprev + (IX)opposite<L>(i) * N + cell) : 0.f);
            } else {
                f[i] = __ldg(a.fprev + (IX)i * N + tgt(i));
            }
        }
        if constexpr (BOX) {
            float w[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) w[i] = f[i];
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (bnf[i]) {
                    const int j = reflect_mask<L>(i, bnf[i]);
#pragma unroll
                    for (int k = 0; k < Q; ++k)
                        if (k == j) f[i] = w[k];
                }
        }
        const bool lo = WALLS && y == 0 && a.bc_lo != BC_PERIODIC;
        const bool hi = WALLS && y == ny - 1 && a.bc_hi != BC_PERIODIC;
        const int kind = lo ? a.bc_lo : a.bc_hi;
        if (lo || hi) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ey(i) != 0 && ((L::ey(i) == 1) == lo)) {
                    if (kind == BC_NOFLUX) f[i] = f[mirror_y<L>(i)];
                    else if (kind == BC_BOUNCE) f[i] = __ldg(a.fprev + (IX)opposite<L>(i) * N + cell);
                }
        }
        // Dirichlet fill (y faces, wall mode 1 or 2): the inward populations are
        // phi_s w_i with w = f^eq(1, u(k - 1)) and phi_s from the others (Sec. 3.2)
        const bool dlo = WM > 0 && y == 0 && a.bc_lo == BC_DIRICHLET;
        const bool dhi = WM > 0 && y == ny - 1 && a.bc_hi == BC_DIRICHLET;
        float dw[Q], dW = 1.f;
        if (dlo || dhi) {
            float up[3] = {0.f, 0.f, 0.f};
            float sp[3];
            sched_row_at(a.sched, a.srow_prev, DIM, sp);
            if (UK == U_FIELD) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) up[d] = __fmul_rn(__ldg(a.ua + (IX)d * N + cell), sp[d]);
            } else if (UK == U_ROW) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) up[d] = __fmul_rn(__ldg(a.ua + d * ny + y), sp[d]);
            }
            const int inward = dlo ? 1 : -1;
            float known = 0.f, wk = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                dw[i] = feq_unit<L>(c, i, up[0], up[1], up[2]);
                if (L::ey(i) == inward) wk += dw[i];
                else known += f[i];
            }
            dW = wk;
            const float ps = ((dlo ? a.phiw_lo : a.phiw_hi) - known) / wk;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ey(i) == inward) f[i] = __fmul_rn(ps, dw[i]);
        }
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (UK == U_FIELD) {
            ux = __fmul_rn(__ldg(a.ua + cell), s_now[0]);
            uy = __fmul_rn(__ldg(a.ua + N + cell), s_now[1]);
            if (DIM == 3) uz = __fmul_rn(__ldg(a.ua + 2 * N + cell), s_now[2]);
        } else if (UK == U_ROW) {
            ux = __fmul_rn(__ldg(a.ua + y), s_now[0]);
            uy = __fmul_rn(__ldg(a.ua + ny + y), s_now[1]);
            if (DIM == 3) uz = __fmul_rn(__ldg(a.ua + 2 * ny + y), s_now[2]);
        }
        const float u[3] = {ux, uy, uz};

        // forward non-equilibrium moments d = M f - m^eq(phi, u(k))
        float m[Q];
        moments<L>(f, m);
        const float phi = m[0];
        float v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = 0.f;
        v[0] = 1.f;
        v[1] = c.meq1;
        v[2] = c.meq2;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            v[3 + 2 * d] = u[d];
            v[4 + 2 * d] = -u[d];
        }
        // MRT-B1/B2 (D2Q9, Eq. 38-39): the u^2 terms of m^eq
        if constexpr (QUAD) {
            const float u2 = fmaf(ux, ux, uy * uy);
            v[1] = fmaf(c.b1, u2, c.meq1);
            v[2] = fmaf(c.b2, u2, c.meq2);
            v[7] = c.g7 * fmaf(ux, ux, -uy * uy);
            v[8] = c.g8 * (ux * uy);
        }
        float dm[Q];
#pragma unroll
        for (int k = 1; k < Q; ++k) dm[k] = fmaf(-phi, v[k], m[k]);
        dm[0] = 0.f;

        // a = M^-T mu = diag(1/|M_r|^2) M mu
        float av[Q];
        moments<L>(mu, av);
#pragma unroll
        for (int k = 0; k < Q; ++k) av[k] *= 1.0f / (float)row_norm2<L>(k);
        // b = S^T a (S of Eq. 31 / A.5: diagonal rates, flux block A, couplings C)
        float b[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) b[k] = c.s[k] * av[k];
#pragma unroll
        for (int bb = 0; bb < DIM; ++bb) {
            float rf = 0.f, rq = 0.f;
#pragma unroll
            for (int aa = 0; aa < DIM; ++aa) {
                rf = fmaf(c.A[aa * DIM + bb], av[3 + 2 * aa], rf);
                rq = fmaf(c.C[aa * DIM + bb], av[3 + 2 * aa], rq);
            }
            b[3 + 2 * bb] = rf;
            b[4 + 2 * bb] += rq;
        }
        float vb = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) vb = fmaf(v[k], b[k], vb);
        float cv[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) cv[k] = av[k] - b[k];
        cv[0] += vb;
        float nu[Q];
        populations<L, false, true>(cv, nu);   // nu = M^T c
        if (!live) continue;

        // velocity partials: u(x, k) = a(x) s(k)  =>  dL/da += s(k) dL/du(k)
        if (DA) {
            float gu[DIM];   // dL/du(k) / phi = b . dv/du
#pragma unroll
            for (int d = 0; d < DIM; ++d) gu[d] = b[3 + 2 * d] - b[4 + 2 * d];
            if constexpr (QUAD) {
                const float q12 = fmaf(c.b1, b[1], c.b2 * b[2]);
                gu[0] += fmaf(2.f * ux, fmaf(c.g7, b[7], q12), c.g8 * uy * b[8]);
                gu[1] += fmaf(2.f * uy, fmaf(-c.g7, b[7], q12), c.g8 * ux * b[8]);
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) a.du_acc[(IX)d * N + cell] = du_old[d] + phi * gu[d] * s_now[d];
        } else if (UK == U_FIELD && a.du_acc != nullptr) {
            // never taken (gradient buffers go to the DA instance); kept because this
            // instance measured faster with it (register allocation)
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                float* p = a.du_acc + (IX)d * N + cell;
                *p += phi * (b[3 + 2 * d] - b[4 + 2 * d]) * s_now[d];
            }
        }
        // parameter partials (FP32 per thread over its rows)
#pragma unroll
        for (int aa = 0; aa < DIM; ++aa)
#pragma unroll
            for (int bb = 0; bb < DIM; ++bb) {
                g[aa * DIM + bb] = fmaf(-av[3 + 2 * aa], dm[3 + 2 * bb], g[aa * DIM + bb]);
                g[DIM * DIM + aa * DIM + bb] = fmaf(-av[3 + 2 * aa], dm[4 + 2 * bb], g[DIM * DIM + aa * DIM + bb]);
            }
#pragma unroll
        for (int k = 1; k < Q; ++k) g[2 * DIM * DIM + k] = fmaf(-av[k], dm[k], g[2 * DIM * DIM + k]);

        // push nu with the transposed wall rules; first the Dirichlet fill's: every
        // other population takes -sum_i w_i nu_i / W over the inward i, which carry
        // nothing further back
        if (dlo || dhi) {
            const int inward = dlo ? 1 : -1;
            float lw = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ey(i) == inward) lw = fmaf(dw[i], nu[i], lw);
            const float r = lw / dW;
#pragma unroll
            for (int i = 0; i < Q; ++i) nu[i] = L::ey(i) == inward ? 0.f : nu[i] - r;
        }
        float* out = a.mu_out;
        if constexpr (BOX) {
            float reg[Q], own[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) reg[k] = own[k] = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int t = bnf[i] ? reflect_mask<L>(i, bnf[i]) : i;   // population whose value i took
#pragma unroll
                for (int k = 0; k < Q; ++k)
                    if (k == t) {
                        if (!bout[k]) reg[k] += nu[i];
                        else if (bbb[k]) own[opposite<L>(k)] += nu[i];
                    }
            }
#pragma unroll
            for (int j = 0; j < Q; ++j)
                if (!bout[j]) out[(IX)j * N + bsrc[j]] = reg[j];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (bout[opposite<L>(k)]) out[(IX)k * N + cell] = own[k];   // k leaves through a wall
            continue;
        }
        if (lo || hi) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (L::ey(i) != 0 && ((L::ey(i) == 1) == lo)) {          // entered from beyond the wall
                    if (kind == BC_NOFLUX) nu[mirror_y<L>(i)] += nu[i];
                    else if (kind == BC_BOUNCE) out[(IX)opposite<L>(i) * N + cell] = nu[i];
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (L::ey(i) != 0 && ((L::ey(i) == 1) == lo)) continue;
                if (kind != BC_BOUNCE && L::ey(i) != 0) out[(IX)i * N + cell] = 0.f;  // left the domain
                out[(IX)i * N + tgt(i)] = nu[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) out[(IX)i * N + tgt(i)] = nu[i];
        }
    }

    // block reduction of the gradient partials (FP32), through shared memory:
    // every thread stores its NG sums as one column of red[NG][256]; then 8 NG
    // threads add 32 consecutive columns of one row each, and NG threads add the
    // 8 segments of their row (a fixed order; about a third of the issue slots of
    // a shuffle tree over NG values)
    __shared__ float red[NG][256];
    __shared__ float seg[NG][8];
#pragma unroll
    for (int j = 0; j < NG; ++j) red[j][threadIdx.x] = g[j];
    __syncthreads();
    if ((int)threadIdx.x < 8 * NG) {
        const int j = threadIdx.x >> 3, sg = threadIdx.x & 7;
        const float* r = &red[j][sg * 32];
        float s = 0.f;
#pragma unroll 8
        for (int c = 0; c < 32; ++c) s += r[(c + sg + 8 * j) & 31];   // staggered start: no bank conflicts
        seg[j][sg] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < NG) {
        float s = 0.f;
#pragma unroll
        for (int sg = 0; sg < 8; ++sg) s += seg[threadIdx.x][sg];
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
        a.partials[threadIdx.x * nb + blk] = s;   // [NG][nblocks]: coalesced in the reduction
    }
}

// Deterministic two-level sum of the per-block partials ([NG][nblocks] in each
// of nslice slices `slice` floats apart, one slice per reverse step since the
// last reduction): pass 2 reduces
// GRAD_CHUNKS contiguous chunks of every row of every slice in parallel, pass 3
// adds the chunk sums in index order to the running totals.
constexpr int GRAD_CHUNKS = 32;

__global__ void __launch_bounds__(256) k_grad_sum2(const float* __restrict__ partials, long long nblocks,
                                                   long long slice, int ng, int nslice, float2* __restrict__ p2)
{
    const int r = blockIdx.x, j = blockIdx.y;
    const long long len = (nblocks + GRAD_CHUNKS - 1) / GRAD_CHUNKS;
    const long long b0 = r * len;
    const long long b1 = b0 + len < nblocks ? b0 + len : nblocks;
    float2 s = make_float2(0.f, 0.f);
    for (int sl = 0; sl < nslice; ++sl) {
        const float* row = partials + (long long)sl * slice + (long long)j * nblocks;
        for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) csum_add(s, row[b]);
    }
    __shared__ float2 red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) csum_merge(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) p2[(long long)j * GRAD_CHUNKS + r] = red[0];
}

__global__ void k_grad_sum3(const float2* __restrict__ p2, int ng, float2* __restrict__ acc)
{
    const int j = threadIdx.x;
    if (j >= ng) return;
    float2 s = acc[j];
    for (int r = 0; r < GRAD_CHUNKS; ++r) csum_merge(s, p2[j * GRAD_CHUNKS + r]);
    acc[j] = s;
}

// Gradients through the initial state B_0 = f^eq(phi0, u(0)):
//   dL/dphi0 = sum_i mu_0,i f^eq_i(1, u),   dL/da += s(0) phi0 sum_i mu_0,i d f^eq_i(1, u) / du
// (= k_i e_i for the equilibria linear in u; MRT-B1/B2 add their u^2 terms)
template <class L, int UK>
__global__ void k_adjoint_init(const AdjArgs a, const float* __restrict__ phi0, float* __restrict__ dphi0)
{
    float s0[3];
    sched_at(a.sched, a.sched_len, 0, L::DIM, s0);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((c / a.nx) % a.ny);
        float ux, uy, uz;
        vel_at_p<UK, L::DIM>(a.ua, a.ncell, a.ny, c, y, s0, ux, uy, uz);
        float gp = 0.f, gu[3] = {0.f, 0.f, 0.f};
        if (L::Q == 9 && (a.c.b1 != 0.f || a.c.g7 != 0.f)) {
            // MRT-B1/B2 (Eq. 38-39): f^eq = M^T diag(1/|M_k|^2) m^eq(phi, u) carries u^2
            // terms, so dL/du = phi0 beta . dm^eq/du with beta = diag(1/|M_k|^2) M mu_0
            float mu[L::Q], fe[L::Q], bt[L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; ++i) mu[i] = __ldg(a.mu_in + (long long)i * a.ncell + c);
            feq_full<L>(a.c, 1.f, ux, uy, uz, fe);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) gp = fmaf(mu[i], fe[i], gp);
#pragma unroll
            for (int k = 0; k < L::Q; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < L::Q; ++i) acc = fmaf((float)L::M(k, i), mu[i], acc);
                bt[k] = acc * (1.0f / (float)row_norm2<L>(k));
            }
            const float q12 = fmaf(a.c.b1, bt[1], a.c.b2 * bt[2]);
            gu[0] = bt[3] - bt[4] + fmaf(2.f * ux, fmaf(a.c.g7, bt[7], q12), a.c.g8 * uy * bt[8]);
            gu[1] = bt[5] - bt[6] + fmaf(2.f * uy, fmaf(-a.c.g7, bt[7], q12), a.c.g8 * ux * bt[8]);
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const float m = __ldg(a.mu_in + (long long)i * a.ncell + c);
                gp = fmaf(m, feq_unit<L>(a.c, i, ux, uy, uz), gp);
                const float k = wclass<L>(i) == 1 ? a.c.ka : (wclass<L>(i) == 2 ? a.c.kd : 0.f);
                gu[0] = fmaf(m * k, (float)L::ex(i), gu[0]);
                gu[1] = fmaf(m * k, (float)L::ey(i), gu[1]);
                gu[2] = fmaf(m * k, (float)L::ez(i), gu[2]);
            }
        }
        dphi0[c] = gp;
        if (UK == U_FIELD && a.du_acc != nullptr) {
            const float p = phi0[c];
            for (int d = 0; d < L::DIM; ++d) a.du_acc[(long long)d * a.ncell + c] += s0[d] * p * gu[d];
        }
    }
}

// mu_N,i = dL/dphi_N for every i (phi_N = sum_i B_N,i)
__global__ void k_adjoint_seed(const float* __restrict__ g, float* __restrict__ mu, long long ncell, int q)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const float v = g[c];
        for (int i = 0; i < q; ++i) mu[(long long)i * ncell + c] = v;
    }
}

static long long adj_blocks(const AdjArgs& a)
{
    return (long long)((a.nx + 255) / 256) * ((a.ny + a.rows - 1) / a.rows) * a.nz;
}

// grad_acc += the per-block partials of nslice slices starting at base, summed in a fixed order
template <class L>
static cudaError_t grad_reduce(const AdjArgs& a, float* base, int nslice, long long slice, cudaStream_t st)
{
    constexpr int NG = ngrad<L>();
    const long long nb = adj_blocks(a);
    float2* p2 = reinterpret_cast<float2*>(base + (long long)ADJ_SLICES * slice);   // slice is even
    k_grad_sum2<<<dim3(GRAD_CHUNKS, NG), 256, 0, st>>>(base, nb, slice, NG, nslice, p2);
    k_grad_sum3<<<1, 64, 0, st>>>(p2, NG, a.grad_acc);
    return cudaGetLastError();
}

template <class L, int UK, typename IX, int WM>
static cudaError_t adj_wm(const AdjArgs& a, cudaStream_t st, bool reduce)
{
    dim3 grid((unsigned)((a.nx + 255) / 256), (unsigned)((a.ny + a.rows - 1) / a.rows), (unsigned)a.nz);
    // the u^2 terms of MRT-B1/B2 (zero coefficients for the other models; with no
    // velocity they vanish)
    constexpr bool QOK = L::Q == 9 && UK != U_NONE;
    const bool quad = QOK && (a.c.b1 != 0.f || a.c.g7 != 0.f);
    if constexpr (UK == U_FIELD) {
        if (a.du_acc != nullptr) {
            if (quad) k_adjoint<L, UK, WM, true, IX, QOK><<<grid, 256, 0, st>>>(a);
            else k_adjoint<L, UK, WM, true, IX, false><<<grid, 256, 0, st>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess || !reduce) return e;
            return grad_reduce<L>(a, a.partials, 1, 0, st);
        }
    }
    if (quad) k_adjoint<L, UK, WM, false, IX, QOK><<<grid, 256, 0, st>>>(a);
    else k_adjoint<L, UK, WM, false, IX, false><<<grid, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !reduce) return e;
    return grad_reduce<L>(a, a.partials, 1, 0, st);
}

template <class L, int UK, typename IX>
static cudaError_t adj_ix(int wmode, const AdjArgs& a, cudaStream_t st, bool reduce)
{
    if (wmode == 2) return adj_wm<L, UK, IX, 2>(a, st, reduce);
    if (wmode == 1) return adj_wm<L, UK, IX, 1>(a, st, reduce);
    return adj_wm<L, UK, IX, 0>(a, st, reduce);
}

template <class L, int UK>
static cudaError_t adj_w(int wmode, const AdjArgs& a, cudaStream_t st, bool reduce)
{
    // 32-bit offsets when every plane (and the velocity planes) fits
    if ((long long)(L::Q + L::DIM) * a.ncell < (1LL << 31)) return adj_ix<L, UK, int>(wmode, a, st, reduce);
    return adj_ix<L, UK, long long>(wmode, a, st, reduce);
}

template <class L>
static cudaError_t adj_u(int uk, int wmode, const AdjArgs& a, cudaStream_t st, bool reduce)
{
    switch (uk) {
        case U_FIELD: return adj_w<L, U_FIELD>(wmode, a, st, reduce);
        case U_ROW: return adj_w<L, U_ROW>(wmode, a, st, reduce);
        default: return adj_w<L, U_NONE>(wmode, a, st, reduce);
    }
}

cudaError_t launch_adjoint(int q, int ukind, int wmode, const AdjArgs& a, cudaStream_t st, bool reduce)
{
    return q == 9 ? adj_u<D2Q9>(ukind, wmode, a, st, reduce) : adj_u<D3Q15>(ukind, wmode, a, st, reduce);
}

cudaError_t launch_grad_reduce(int q, const AdjArgs& a, float* base, int nslice, long long slice, cudaStream_t st)
{
    return q == 9 ? grad_reduce<D2Q9>(a, base, nslice, slice, st) : grad_reduce<D3Q15>(a, base, nslice, slice, st);
}

// Floats of one slice of block partials ([NG][nblocks]), rounded up to an even
// count (8-byte aligned slices).
long long adjoint_slice_size(int q, long long nx, long long ny, long long nz, int sms)
{
    const int rows = adjoint_rows(nx, ny, nz, sms);
    const long long nb = ((nx + 255) / 256) * ((ny + rows - 1) / rows) * nz;
    const long long f = nb * (q == 9 ? ngrad<D2Q9>() : ngrad<D3Q15>());
    return (f + 1) & ~1LL;
}

long long adjoint_partials_size(int q, long long nx, long long ny, long long nz, int sms)
{
    // ADJ_SLICES slices, then the [NG][GRAD_CHUNKS] float2 chunk sums
    return ADJ_SLICES * adjoint_slice_size(q, nx, ny, nz, sms) +
           2LL * GRAD_CHUNKS * (q == 9 ? ngrad<D2Q9>() : ngrad<D3Q15>());
}

int adjoint_ngrad(int q) { return q == 9 ? ngrad<D2Q9>() : ngrad<D3Q15>(); }

template <class L>
static cudaError_t init_u(int uk, const AdjArgs& a, const float* phi0, float* dphi0, cudaStream_t st)
{
    long long b = (a.ncell + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    switch (uk) {
        case U_FIELD: k_adjoint_init<L, U_FIELD><<<(int)b, 256, 0, st>>>(a, phi0, dphi0); break;
        case U_ROW: k_adjoint_init<L, U_ROW><<<(int)b, 256, 0, st>>>(a, phi0, dphi0); break;
        default: k_adjoint_init<L, U_NONE><<<(int)b, 256, 0, st>>>(a, phi0, dphi0); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init(int q, int ukind, const AdjArgs& a, const float* phi0, float* dphi0,
                                cudaStream_t st)
{
    return q == 9 ? init_u<D2Q9>(ukind, a, phi0, dphi0, st) : init_u<D3Q15>(ukind, a, phi0, dphi0, st);
}

cudaError_t launch_adjoint_seed(const float* g, float* mu, long long ncell, int q, cudaStream_t st)
{
    long long b = (ncell + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_adjoint_seed<<<(int)b, 256, 0, st>>>(g, mu, ncell, q);
    return cudaGetLastError();
}

}  // namespace lbm
