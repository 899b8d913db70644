// D2Q9 step for the 16-bit offset storage with TMA staging of the source rows.
//
// A CTA of 128 threads walks down a range of rows of a 256-column strip of the
// grid, one row at a time. Grid row r enters a ring of shared-memory stages through
// tensor copies (cp.async.bulk.tensor) that one thread issues: the nine offset
// planes of row r as one (256, 1, 9) box plus 8-column halo boxes on both
// sides, and phi and the two velocity factors of row r as (256, 1) boxes plus
// 4-column halos. The copies complete on an mbarrier per stage. Node row y
// needs rows y - 1, y, y + 1 (all of phi and u for the decode, and plane i at
// row y - e_iy); while the threads compute it from shared memory, the copies
// of the next rows are in flight, so the loads cost no registers and their
// latency hides behind the arithmetic. The arithmetic per node pair is the one
// of k_step_pair_d2q9 (paired FP32 decode, collide_pair, offsets stored as
// 32-bit pairs). CTA (s, b) walks strip s over the b-th of gridDim.y equal row
// ranges; one wave of CTAs covers the grid.
//
// Every wait on an mbarrier is bounded: on time-out the CTA latches
// LBM_E_TIMEOUT in the status word, stops computing and issuing, waits
// (bounded) for the copies it issued, and returns.
#pragma once
#include "lbm_pair.cuh"
#include "../../include/lbm_cde.h"

namespace lbm {

constexpr int TMA_W = 256;    // strip width in nodes (one box per plane row)
// Per instantiation: R grid rows computed per iteration by 128 R threads (128
// node pairs per row) and a ring of NS >= R + 2 stages (R + 2 rows in use, the
// rest in flight). Launch vec 7: R = 2, NS = 6; vec 8: R = 1, NS = 4.
template <int R, int NS>
struct TmaShape {
    static_assert(NS >= R + 2, "the ring must hold the R + 2 rows one iteration reads");
    static constexpr int threads = 128 * R;
};
// stage layout in bytes; every copy destination is 128-byte aligned
constexpr int TS_G = 0;                       // [9][256] offsets
constexpr int TS_GL = TS_G + 9 * TMA_W * 2;   // [9][8] columns xs - 8 .. xs - 1
constexpr int TS_GR = TS_GL + 256;            // [9][8] columns xs + 256 .. xs + 263
constexpr int TS_P = TS_GR + 256;             // [256] phi
constexpr int TS_PL = TS_P + TMA_W * 4;       // [4] columns xs - 4 .. xs - 1
constexpr int TS_PR = TS_PL + 128;            // [4] columns xs + 256 .. xs + 259
constexpr int TS_U = TS_PR + 128;             // [2][256] velocity factors
constexpr int TS_UL = TS_U + 2 * TMA_W * 4;   // [2][4]
constexpr int TS_UR = TS_UL + 128;            // [2][4]
constexpr int TS_BYTES = TS_UR + 128;         // 8704 bytes per stage
constexpr int tma_smem(int ns) { return ns * TS_BYTES + ns * 8; }   // + one mbarrier per stage
constexpr long long TMA_DRAIN_LIMIT = 4000000000LL;         // clock64 cycles (about 2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase of the given parity for at most `limit` SM cycles (0: gives
// up without looking); false, with LBM_E_TIMEOUT latched in status, on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* status, long long limit)
{
    const long long t0 = clock64();
    while (clock64() - t0 < limit)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicCAS(status, 0, (int)LBM_E_TIMEOUT);
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* m, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* m, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// (v(x0 - 1), v(x0)), (v(x0), v(x0 + 1)), (v(x0 + 1), v(x0 + 2)) of one staged FP32 row
__device__ __forceinline__ void stage_window(const unsigned char* st, int off, int offl, int offr, int t,
                                             float2 (&w)[3])
{
    const float* row = reinterpret_cast<const float*>(st + off);
    const float2 c = *reinterpret_cast<const float2*>(row + 2 * t);
    const float l = t == 0 ? reinterpret_cast<const float*>(st + offl)[3] : row[2 * t - 1];
    const float r = t == TMA_W / 2 - 1 ? reinterpret_cast<const float*>(st + offr)[0] : row[2 * t + 2];
    w[0] = make_float2(l, c.x);
    w[1] = c;
    w[2] = make_float2(c.y, r);
}

template <int STORE, int UK, bool WALLS, int TMA_R, int TMA_NS>
__global__ void __launch_bounds__(TmaShape<TMA_R, TMA_NS>::threads)
    k_step_tma_d2q9(const StepArgs a, const __grid_constant__ TmaMaps m)
{
    using P = Pair<STORE>;
    using T2 = typename P::T2;
    using L = D2Q9;
    extern __shared__ __align__(128) unsigned char sm[];
    const int nx = a.nx, ny = a.ny;
    const int t = threadIdx.x;
    const int tp = t % (TMA_W / 2);   // node pair (x0 = xs + 2 tp) within the strip
    const int rr = t / (TMA_W / 2);   // row within the iteration
    const uint32_t bar0 = smem_addr(sm + TMA_NS * TS_BYTES);
    if (t == 0) {
        for (int s = 0; s < TMA_NS; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    constexpr uint32_t TX = 9 * TMA_W * 2 + 2 * 9 * 8 * 2 + TMA_W * 4 + 2 * 16 +
                            (UK == U_FIELD ? 2 * TMA_W * 4 + 2 * 2 * 4 * 4 : 0);
    const Coef& c = a.c;
    float s_now[3], s_prev[3];
    sched_row_at(a.sched, a.srow_now, 2, s_now);
    sched_row_at(a.sched, a.srow_prev, 2, s_prev);
    // decode slopes k_i s_d(k - 1) of the axis (a) and diagonal (d) populations: the
    // schedule factor folded in, so a diagonal population costs two paired FMAs
    const float kax = __fmul_rn(c.ka, s_prev[0]), kay = __fmul_rn(c.ka, s_prev[1]);
    const float kdx = __fmul_rn(c.kd, s_prev[0]), kdy = __fmul_rn(c.kd, s_prev[1]);
    T2* __restrict__ dst = static_cast<T2*>(a.dst);
    const int NP = (int)(a.ncell / 2), nxp = nx / 2;

    // strip blockIdx.x, rows [ya, yb) of block row blockIdx.y: neighbouring strips
    // run the same rows at the same time, so their halo columns meet in L2
    const int xs = (int)blockIdx.x * TMA_W;
    const int ya = (int)((long long)blockIdx.y * ny / gridDim.y);
    const int yb = (int)((long long)(blockIdx.y + 1) * ny / gridDim.y);
    const unsigned seq = 0;    // row q of the walk sits in stage q % NS, completion parity (q / NS) & 1
    unsigned issued = 0;       // (thread 0) rows issued so far
    bool ok = true;
    if (ya < yb) {
        const int nrow = yb - ya + 2;   // grid rows ya - 1 .. yb (periodic)
        const int xl8 = xs == 0 ? nx - 8 : xs - 8, xl4 = xs == 0 ? nx - 4 : xs - 4;
        const int xr = xs + TMA_W == nx ? 0 : xs + TMA_W;
        auto issue = [&](int j) {      // thread 0: stage grid row ya - 1 + j
            const unsigned q = seq + j;
            unsigned char* st = sm + (q % TMA_NS) * TS_BYTES;
            const uint32_t bar = bar0 + 8 * (q % TMA_NS);
            int yr = ya - 1 + j;
            yr = yr < 0 ? yr + ny : (yr >= ny ? yr - ny : yr);
            mbar_expect_tx(bar, TX);
            tma_load_3d(smem_addr(st + TS_G), &m.g, xs, yr, 0, bar);
            tma_load_3d(smem_addr(st + TS_GL), &m.gh, xl8, yr, 0, bar);
            tma_load_3d(smem_addr(st + TS_GR), &m.gh, xr, yr, 0, bar);
            tma_load_2d(smem_addr(st + TS_P), &m.p, xs, yr, bar);
            tma_load_2d(smem_addr(st + TS_PL), &m.ph, xl4, yr, bar);
            tma_load_2d(smem_addr(st + TS_PR), &m.ph, xr, yr, bar);
            if (UK == U_FIELD) {
                tma_load_3d(smem_addr(st + TS_U), &m.u, xs, yr, 0, bar);
                tma_load_3d(smem_addr(st + TS_UL), &m.uh, xl4, yr, 0, bar);
                tma_load_3d(smem_addr(st + TS_UR), &m.uh, xr, yr, 0, bar);
            }
            issued = q + 1;
        };
        auto wait = [&](int j) {
            const unsigned q = seq + j;
            ok = ok && mbar_wait_bounded(bar0 + 8 * (q % TMA_NS), (q / TMA_NS) & 1u, a.status, a.spin_limit);
        };
        if (t == 0)
            for (int j = 0; j < TMA_NS && j < nrow; ++j) issue(j);
        int waited = 0;   // staged rows 0 .. waited - 1 are complete
        for (int y0 = ya; y0 < yb; y0 += TMA_R) {
            const int j0 = y0 - ya + 1;                                   // walk index of row y0
            const int jl = j0 + TMA_R < nrow - 1 ? j0 + TMA_R : nrow - 1;   // last staged row read
            for (; waited <= jl; ++waited) wait(waited);
            const int y = y0 + rr, j = j0 + rr;
            if (ok && y < yb) {
                // staged rows by e_y + 1: y + 1, y, y - 1
                const unsigned char* S[3] = {sm + ((seq + j + 1) % TMA_NS) * TS_BYTES,
                                             sm + ((seq + j) % TMA_NS) * TS_BYTES,
                                             sm + ((seq + j - 1) % TMA_NS) * TS_BYTES};
                // phi and the velocity factors a (u = a s) of the source windows
                float2 Ps[3][3], Ax[3][3], Ay[3][3];
                float2 axo = sp2(0.f), ayo = sp2(0.f);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    stage_window(S[r], TS_P, TS_PL, TS_PR, tp, Ps[r]);
                    if (UK == U_FIELD) {
                        stage_window(S[r], TS_U, TS_UL, TS_UR, tp, Ax[r]);
                        stage_window(S[r], TS_U + TMA_W * 4, TS_UL + 16, TS_UR + 16, tp, Ay[r]);
                        if (r == 1) {
                            axo = Ax[1][1];
                            ayo = Ay[1][1];
                        }
                    } else if (UK == U_ROW) {
                        const int yr = r == 0 ? (y + 1 == ny ? 0 : y + 1) : (r == 1 ? y : (y == 0 ? ny - 1 : y - 1));
                        const float ax = __ldg(a.ua + yr), ay = __ldg(a.ua + ny + yr);
#pragma unroll
                        for (int k = 0; k < 3; ++k) Ax[r][k] = sp2(ax), Ay[r][k] = sp2(ay);
                        if (r == 1) {
                            axo = sp2(ax);
                            ayo = sp2(ay);
                        }
                    }
                }
                // pull and decode f_i = g_i(s) + phi(s) f^eq_i(1, u(s, k-1))
                float2 f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ex = L::ex(i), r = L::ey(i) + 1, cp = 1 - ex;
                    const unsigned* gw = reinterpret_cast<const unsigned*>(S[r] + TS_G + i * TMA_W * 2);
                    unsigned w = gw[tp];
                    if (ex > 0) {
                        const unsigned lo = tp == 0 ? reinterpret_cast<const unsigned*>(S[r] + TS_GL + i * 16)[3]
                                                   : gw[tp - 1];
                        w = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(lo), QuadH<STORE>::as_t2(w)));
                    } else if (ex < 0) {
                        const unsigned hi = tp == TMA_W / 2 - 1 ? reinterpret_cast<const unsigned*>(S[r] + TS_GR + i * 16)[0]
                                                           : gw[tp + 1];
                        w = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(w), QuadH<STORE>::as_t2(hi)));
                    }
                    // f^eq_i / phi = w_i + k_i e_i . a s(k - 1)
                    const int wc = wclass<L>(i), ey = L::ey(i);
                    float2 e = sp2(wc == 0 ? c.w0 : (wc == 1 ? c.wa : c.wd));
                    if (UK != U_NONE && wc != 0) {
                        const float sx = wc == 1 ? kax : kdx, sy = wc == 1 ? kay : kdy;
                        if (ex != 0) e = fma2(sp2(ex > 0 ? sx : -sx), Ax[r][cp], e);
                        if (ey != 0) e = fma2(sp2(ey > 0 ? sy : -sy), Ay[r][cp], e);
                    }
                    f[i] = fma2(Ps[r][cp], e, P::to_f(QuadH<STORE>::as_t2(w)));
                }
                const int cellp = y * nxp + (xs >> 1) + tp;
                if (WALLS) {
                    const bool lo = (y == 0) && a.bc_lo != BC_PERIODIC;
                    const bool hi = (y == ny - 1) && a.bc_hi != BC_PERIODIC;
                    if (lo || hi) {
                        const int kind = lo ? a.bc_lo : a.bc_hi;
                        const int inward = lo ? 1 : -1;
                        const float2 uxp = mul2(axo, sp2(s_prev[0])), uyp = mul2(ayo, sp2(s_prev[1]));
                        if (kind == BC_NOFLUX) {
#pragma unroll
                            for (int i = 0; i < 9; ++i)
                                if (L::ey(i) == inward) f[i] = f[mirror_y<L>(i)];
                        } else if (kind == BC_BOUNCE) {
#pragma unroll
                            for (int i = 0; i < 9; ++i)
                                if (L::ey(i) == inward) {
                                    const int o = opposite<L>(i);
                                    const unsigned w =
                                        reinterpret_cast<const unsigned*>(S[1] + TS_G + o * TMA_W * 2)[tp];
                                    const float2 g = P::to_f(QuadH<STORE>::as_t2(w));
                                    f[i] = fma2(Ps[1][1], feq_unit_pair(c, o, uxp, uyp), g);
                                }
                        } else {   // Dirichlet
                            float2 known = sp2(0.f), wk = sp2(0.f);
#pragma unroll
                            for (int i = 0; i < 9; ++i) {
                                if (L::ey(i) == inward) wk = add2(wk, feq_unit_pair(c, i, uxp, uyp));
                                else known = add2(known, f[i]);
                            }
                            const float phiw = lo ? a.phiw_lo : a.phiw_hi;
                            const float2 ps = make_float2((phiw - known.x) / wk.x, (phiw - known.y) / wk.y);
#pragma unroll
                            for (int i = 0; i < 9; ++i)
                                if (L::ey(i) == inward) f[i] = mul2(ps, feq_unit_pair(c, i, uxp, uyp));
                        }
                    }
                }
                float2 uxn = sp2(0.f), uyn = sp2(0.f);
                if (UK != U_NONE) {
                    uxn = mul2(axo, sp2(s_now[0]));
                    uyn = mul2(ayo, sp2(s_now[1]));
                }
                const float2 phi = collide_pair(f, uxn, uyn, c);
#pragma unroll
                for (int i = 0; i < 9; ++i) dst[i * NP + cellp] = P::from_f(f[i]);
                *reinterpret_cast<float2*>(a.phi_dst + 2 * cellp) = phi;
            }
            // every thread is done with the stages of rows y0 - 1 .. y0 + R - 2; ok becomes CTA-uniform
            ok = __syncthreads_and(ok) != 0;
            if (t == 0 && ok)
                for (int r = 0; r < TMA_R; ++r)
                    if (j0 - 1 + r + TMA_NS < nrow) issue(j0 - 1 + r + TMA_NS);
        }
    }
    if (t == 0 && !ok) {
        // bounded wait for this CTA's copies still in flight before its shared memory is released
        for (unsigned q = issued > TMA_NS ? issued - TMA_NS : 0; q < issued; ++q)
            mbar_wait_bounded(bar0 + 8 * (q % TMA_NS), (q / TMA_NS) & 1u, nullptr, TMA_DRAIN_LIMIT);
    }
}

// One wave of CTAs: strips x block rows, with as many block rows as the
// resident CTAs (per SM x SMs) allow per strip.
template <int STORE, int UK, bool WALLS, int R, int NS>
cudaError_t launch_tma_d2q9(const StepArgs& a, cudaStream_t st)
{
    constexpr int threads = TmaShape<R, NS>::threads, smem = tma_smem(NS);
    static int resident_by_dev[64] = {0};   // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    int& resident = resident_by_dev[dev & 63];
    if (resident == 0) {
        int nsm = 0, per_sm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step_tma_d2q9<STORE, UK, WALLS, R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_tma_d2q9<STORE, UK, WALLS, R, NS>, threads,
                                                      smem);
        resident = (nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
    }
    const int nstrip = a.nx / TMA_W;
    int nb = resident / nstrip;
    nb = nb < 1 ? 1 : (nb > a.ny ? a.ny : nb);
    k_step_tma_d2q9<STORE, UK, WALLS, R, NS><<<dim3((unsigned)nstrip, (unsigned)nb), threads, smem, st>>>(a, *a.tma);
    return cudaGetLastError();
}

}  // namespace lbm
