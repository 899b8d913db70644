// D3Q15 step for the 16-bit offset storage with TMA staging of the source rows
// (Appendix A lattice; arithmetic of k_step_pair_d3q15).
//
// A CTA of 64 R threads owns a 128-column strip of one z plane and walks down
// a range of its rows, R rows per iteration, one node pair per thread. Node
// (x, y, z) pulls population i from (x - e_ix, y - e_iy, z - e_iz), so row y
// reads the grid rows y - 1, y, y + 1 of the planes z - 1, z, z + 1. A stage of
// the shared-memory ring holds one grid row y' at the three planes, and for
// each plane z' = z - e_z only what the pulls read there: the five offset planes
// with that e_z (e_z = 0: rest, +-x, +-y; e_z = +-1: the z axis and four
// corners) with 8-column halos where e_x != 0, phi and the three velocity
// factors with 4-column halos. Tensor copies (cp.async.bulk.tensor, issued by
// one thread) fill a stage and complete on its mbarrier; R + 2 stages are read
// per iteration while the next rows are in flight. Every offset, phi and
// velocity value a node pair decodes comes from shared memory: the up to 15
// gathers per value of the direct-load kernel cost no registers and no
// global-load latency here.
//
// Every wait on an mbarrier is bounded (lbm_cde_set_wait_limit): on time-out
// the CTA latches LBM_E_TIMEOUT in the status word, stops computing and
// issuing, waits (bounded) for the copies it issued, and returns.
#pragma once
#include "lbm_pair_d3q15.cuh"
#include "lbm_tma_d2q9.cuh"

namespace lbm {

constexpr int T3_W = 128;     // strip width in nodes
constexpr int T3_TP = T3_W / 2;   // node pairs (threads) per row

// Stage layout in bytes (every copy destination 128-byte aligned). Slot sz =
// e_z + 1 holds plane z - e_z. Within a slot the five offset planes are kept in
// the local order lslot(i): e_z = 0: 0, 1, 2, 3, 4; e_z = +1: 5, 7, 8, 9, 10;
// e_z = -1: 6, 11, 12, 13, 14 (one box for plane 5 or 6, one for the corners).
constexpr int T3_G = 0;                          // [3 slots][5][128] u16
constexpr int T3_GH = T3_G + 3 * 5 * T3_W * 2;   // [3 slots][2 sides] 128-byte chunks: [<=4][8] u16
constexpr int T3_P = T3_GH + 3 * 2 * 128;        // [3 slots][128] phi
constexpr int T3_PH = T3_P + 3 * T3_W * 4;       // [3 slots][2 sides] chunks: [4] phi
constexpr int T3_U = T3_PH + 3 * 2 * 128;        // [3 slots][3 comps][128] velocity factors
constexpr int T3_UH = T3_U + 3 * 3 * T3_W * 4;   // [3 slots][2 sides] chunks: [3][4]
constexpr int T3_BYTES = T3_UH + 3 * 2 * 128;    // 12288 bytes per stage
__host__ __device__ constexpr int tma3_smem(int ns) { return ns * T3_BYTES + ns * 8; }

// Bytes one stage receives (the mbarrier's transaction count).
__host__ __device__ constexpr uint32_t t3_tx(bool field)
{
    return 3 * 5 * T3_W * 2 +                          // offsets
           2 * (2 * 8 * 2) + 2 * 2 * (4 * 8 * 2) +     // offset halos: +-x planes, corner planes
           3 * T3_W * 4 + 3 * 2 * 16 +                 // phi
           (field ? 3 * 3 * T3_W * 4 + 3 * 2 * 48 : 0);   // velocity factors
}

// local position of population i among the five offset planes of its slot
__host__ __device__ constexpr int t3_local(int i)
{
    return D3Q15::ez(i) == 0 ? i : ((i == 5 || i == 6) ? 0 : (D3Q15::ez(i) > 0 ? i - 6 : i - 10));
}
// position of population i (e_x != 0) within its slot's halo box: the x axis
// pair (planes 1, 2) in the e_z = 0 slot, the four corners otherwise
__host__ __device__ constexpr int t3_halo(int i)
{
    return D3Q15::ez(i) == 0 ? i - 1 : (D3Q15::ez(i) > 0 ? i - 7 : i - 11);
}

// (v(x0 - 1), v(x0)), (v(x0), v(x0 + 1)) or (v(x0 + 1), v(x0 + 2)) (e_x = +1, 0,
// -1) of a staged FP32 row of the strip, with the 4-column halos
__device__ __forceinline__ float2 t3_window(const float* row, const float* hl, const float* hr, int tp, int ex)
{
    const float2 c = *reinterpret_cast<const float2*>(row + 2 * tp);
    if (ex == 0) return c;
    if (ex > 0) return make_float2(tp == 0 ? hl[3] : row[2 * tp - 1], c.x);
    return make_float2(c.y, tp == T3_TP - 1 ? hr[0] : row[2 * tp + 2]);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* m, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Needs nx % 128 == 0, 18 ncell < 2^31 (int offsets), a 16-byte aligned velocity
// field and the tensor maps of the source buffer (checked by the launcher).
template <int STORE, int UK, bool WALLS, int TR, int TNS>
__global__ void __launch_bounds__(T3_TP * TR)
    k_step_tma_d3q15(const StepArgs a, const __grid_constant__ TmaMaps15 m)
{
    static_assert(TNS >= TR + 2, "the ring must hold the R + 2 rows one iteration reads");
    using P = Pair<STORE>;
    using T2 = typename P::T2;
    using L = D3Q15;
    constexpr float SC = STORE == ST_F16 ? F16_SCALE : 1.f;   // working units (k_step_pair_d3q15)
    extern __shared__ __align__(128) unsigned char sm[];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const int tp = t % T3_TP;   // node pair (x0 = xs + 2 tp) within the strip
    const int rr = t / T3_TP;   // row within the iteration
    const uint32_t bar0 = smem_addr(sm + TNS * T3_BYTES);
    if (t == 0) {
        for (int s = 0; s < TNS; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    constexpr uint32_t TX = t3_tx(UK == U_FIELD);
    const Coef& c = a.c;
    float s_now[3], s_prev[3];
    sched_row_at(a.sched, a.srow_now, 3, s_now);
    sched_row_at(a.sched, a.srow_prev, 3, s_prev);
    const float w0 = c.w0 * SC, wa = c.wa * SC, wd = c.wd * SC;   // exact (power of two)
    const float ka = c.ka * SC, kd = c.kd * SC;
    float kas[3], kds[3];   // decode slopes with the schedule factor of u(k - 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        kas[d] = __fmul_rn(ka, s_prev[d]);
        kds[d] = __fmul_rn(kd, s_prev[d]);
    }
    const T2* __restrict__ src = static_cast<const T2*>(a.src);
    T2* __restrict__ dst = static_cast<T2*>(a.dst);
    const int NP = (int)(a.ncell / 2), nxp = nx / 2;

    // strip blockIdx.x of plane blockIdx.y, rows [ya, yb) of range blockIdx.z
    const int xs = (int)blockIdx.x * T3_W;
    const int z = (int)blockIdx.y;
    const int zsl[3] = {z + 1 == nz ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};   // plane of slot e_z + 1
    const int ya = (int)((long long)blockIdx.z * ny / gridDim.z);
    const int yb = (int)((long long)(blockIdx.z + 1) * ny / gridDim.z);
    unsigned issued = 0;   // (thread 0) rows issued so far; row q of the walk sits in stage q % TNS
    bool ok = true;
    if (ya < yb) {
        const int nrow = yb - ya + 2;   // grid rows ya - 1 .. yb (periodic)
        const int xl8 = xs == 0 ? nx - 8 : xs - 8, xl4 = xs == 0 ? nx - 4 : xs - 4;
        const int xr = xs + T3_W == nx ? 0 : xs + T3_W;
        auto issue = [&](int j) {      // thread 0: stage grid row ya - 1 + j at the three planes
            const unsigned q = (unsigned)j;
            unsigned char* st = sm + (q % TNS) * T3_BYTES;
            const uint32_t bar = bar0 + 8 * (q % TNS);
            int yr = ya - 1 + j;
            yr = yr < 0 ? yr + ny : (yr >= ny ? yr - ny : yr);
            mbar_expect_tx(bar, TX);
#pragma unroll
            for (int sz = 0; sz < 3; ++sz) {
                const int zp = zsl[sz];
                unsigned char* g = st + T3_G + sz * 5 * T3_W * 2;
                unsigned char* gl = st + T3_GH + (2 * sz) * 128;
                unsigned char* gr = gl + 128;
                if (sz == 1) {
                    tma_load_4d(smem_addr(g), &m.gA, xs, yr, zp, 0, bar);
                    tma_load_4d(smem_addr(gl), &m.hA, xl8, yr, zp, 1, bar);
                    tma_load_4d(smem_addr(gr), &m.hA, xr, yr, zp, 1, bar);
                } else {
                    const int pz = sz == 2 ? 5 : 6, pc = sz == 2 ? 7 : 11;   // z-axis plane, first corner
                    tma_load_4d(smem_addr(g), &m.gB, xs, yr, zp, pz, bar);
                    tma_load_4d(smem_addr(g + T3_W * 2), &m.gC, xs, yr, zp, pc, bar);
                    tma_load_4d(smem_addr(gl), &m.hC, xl8, yr, zp, pc, bar);
                    tma_load_4d(smem_addr(gr), &m.hC, xr, yr, zp, pc, bar);
                }
                unsigned char* p = st + T3_P + sz * T3_W * 4;
                unsigned char* pl = st + T3_PH + (2 * sz) * 128;
                tma_load_3d(smem_addr(p), &m.p, xs, yr, zp, bar);
                tma_load_3d(smem_addr(pl), &m.ph, xl4, yr, zp, bar);
                tma_load_3d(smem_addr(pl + 128), &m.ph, xr, yr, zp, bar);
                if (UK == U_FIELD) {
                    unsigned char* u = st + T3_U + sz * 3 * T3_W * 4;
                    unsigned char* ul = st + T3_UH + (2 * sz) * 128;
                    tma_load_4d(smem_addr(u), &m.u, xs, yr, zp, 0, bar);
                    tma_load_4d(smem_addr(ul), &m.uh, xl4, yr, zp, 0, bar);
                    tma_load_4d(smem_addr(ul + 128), &m.uh, xr, yr, zp, 0, bar);
                }
            }
            issued = q + 1;
        };
        auto wait = [&](int j) {
            const unsigned q = (unsigned)j;
            ok = ok && mbar_wait_bounded(bar0 + 8 * (q % TNS), (q / TNS) & 1u, a.status, a.spin_limit);
        };
        if (t == 0)
            for (int j = 0; j < TNS && j < nrow; ++j) issue(j);
        int waited = 0;   // staged rows 0 .. waited - 1 are complete
        for (int y0 = ya; y0 < yb; y0 += TR) {
            const int j0 = y0 - ya + 1;                                 // walk index of row y0
            const int jl = j0 + TR < nrow - 1 ? j0 + TR : nrow - 1;     // last staged row read
            for (; waited <= jl; ++waited) wait(waited);
            const int y = y0 + rr, j = j0 + rr;
            if (ok && y < yb) {
                // staged rows by e_y + 1: y + 1, y, y - 1
                const unsigned char* S[3] = {sm + ((j + 1) % TNS) * T3_BYTES, sm + (j % TNS) * T3_BYTES,
                                             sm + ((j - 1) % TNS) * T3_BYTES};
                float2 f[15];
#pragma unroll
                for (int i = 0; i < 15; ++i) {
                    const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i), sz = ez + 1;
                    const unsigned char* st = S[ey + 1];
                    // offsets of the pair (x0 - e_x, x0 + 1 - e_x) as one 32-bit word
                    const unsigned* gw = reinterpret_cast<const unsigned*>(st + T3_G + (sz * 5 + t3_local(i)) * T3_W * 2);
                    unsigned w = gw[tp];
                    if (ex > 0) {
                        const int hb = 2 * sz, hi = t3_halo(i);
                        const unsigned lo = tp == 0 ? reinterpret_cast<const unsigned*>(st + T3_GH + hb * 128 + hi * 16)[3]
                                                    : gw[tp - 1];
                        w = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(lo), QuadH<STORE>::as_t2(w)));
                    } else if (ex < 0) {
                        const int hb = 2 * sz + 1, hi = t3_halo(i);
                        const unsigned up = tp == T3_TP - 1 ? reinterpret_cast<const unsigned*>(st + T3_GH + hb * 128 + hi * 16)[0]
                                                            : gw[tp + 1];
                        w = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(w), QuadH<STORE>::as_t2(up)));
                    }
                    const float* prow = reinterpret_cast<const float*>(st + T3_P + sz * T3_W * 4);
                    const float* phl = reinterpret_cast<const float*>(st + T3_PH + (2 * sz) * 128);
                    const float2 ps = t3_window(prow, phl, phl + 32, tp, ex);
                    const int wc = wclass<L>(i);
                    float2 e = sp2(wc == 0 ? w0 : (wc == 1 ? wa : wd));
                    if (UK == U_FIELD) {
                        const float* ks = wc == 1 ? kas : kds;
                        const int ed[3] = {ex, ey, ez};
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (ed[d] == 0) continue;
                            const float* urow = reinterpret_cast<const float*>(st + T3_U + (sz * 3 + d) * T3_W * 4);
                            const float* uhl = reinterpret_cast<const float*>(st + T3_UH + (2 * sz) * 128) + 4 * d;
                            const float2 ad = t3_window(urow, uhl, uhl + 32, tp, ex);
                            e = fma2(sp2(ed[d] > 0 ? ks[d] : -ks[d]), ad, e);
                        }
                    } else if (UK == U_ROW && wc != 0) {
                        const int yr = ey == 0 ? y : (ey > 0 ? (y == 0 ? ny - 1 : y - 1) : (y + 1 == ny ? 0 : y + 1));
                        const float ux = __fmul_rn(__ldg(a.ua + yr), s_prev[0]);
                        const float uy = __fmul_rn(__ldg(a.ua + ny + yr), s_prev[1]);
                        const float uz = __fmul_rn(__ldg(a.ua + 2 * ny + yr), s_prev[2]);
                        e = sp2(fmaf(wc == 1 ? ka : kd, e_dot<L>(i, ux, uy, uz), wc == 1 ? wa : wd));
                    }
                    f[i] = fma2(ps, e, P::to_f_raw(QuadH<STORE>::as_t2(w)));
                }
                const int cellp = ((z * ny + y) * nx + xs) / 2 + tp;
                // own velocity factors a(x0), a(x0 + 1)
                float2 ao[3] = {sp2(0.f), sp2(0.f), sp2(0.f)};
                if (UK == U_FIELD) {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        ao[d] = *reinterpret_cast<const float2*>(S[1] + T3_U + (3 + d) * T3_W * 4 + 8 * tp);
                } else if (UK == U_ROW) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) ao[d] = sp2(__ldg(a.ua + d * ny + y));
                }
                if (WALLS) {
                    const bool lo = (y == 0) && a.bc_lo != BC_PERIODIC;
                    const bool hi = (y == ny - 1) && a.bc_hi != BC_PERIODIC;
                    if (lo || hi) {
                        const int kind = lo ? a.bc_lo : a.bc_hi;
                        const int inward = lo ? 1 : -1;   // e_y of the populations entering from the wall
                        float2 up[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) up[d] = mul2(ao[d], sp2(s_prev[d]));
                        if (kind == BC_NOFLUX) {
#pragma unroll
                            for (int i = 0; i < 15; ++i)
                                if (L::ey(i) == inward) f[i] = f[mirror_y<L>(i)];
                        } else if (kind == BC_BOUNCE) {
                            // the node's own reversed populations: their planes are not all
                            // staged at this node's plane, so they come from global memory
                            const float2 po = *reinterpret_cast<const float2*>(S[1] + T3_P + 1 * T3_W * 4 + 8 * tp);
#pragma unroll
                            for (int i = 0; i < 15; ++i)
                                if (L::ey(i) == inward) {
                                    const int o = opposite<L>(i);
                                    const float2 g = P::to_f_raw(ldg_pair(src + o * NP + cellp));
                                    f[i] = fma2(po, feq_unit_pair15(w0, wa, wd, ka, kd, o, up[0], up[1], up[2]), g);
                                }
                        } else {   // Dirichlet
                            float2 known = sp2(0.f), wk = sp2(0.f);
#pragma unroll
                            for (int i = 0; i < 15; ++i) {
                                if (L::ey(i) == inward) wk = add2(wk, feq_unit_pair15(w0, wa, wd, ka, kd, i, up[0], up[1], up[2]));
                                else known = add2(known, f[i]);
                            }
                            const float phiw = (lo ? a.phiw_lo : a.phiw_hi) * SC;
                            const float2 ps = make_float2((phiw - known.x) / wk.x, (phiw - known.y) / wk.y);
#pragma unroll
                            for (int i = 0; i < 15; ++i)
                                if (L::ey(i) == inward) f[i] = mul2(ps, feq_unit_pair15(w0, wa, wd, ka, kd, i, up[0], up[1], up[2]));
                        }
                    }
                }
                float2 un[3] = {sp2(0.f), sp2(0.f), sp2(0.f)};
                if (UK != U_NONE) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) un[d] = mul2(ao[d], sp2(s_now[d]));
                }
                const float2 phi = collide_d3q15<float2, true>(f, un[0], un[1], un[2], c);
#pragma unroll
                for (int i = 0; i < 15; ++i) dst[i * NP + cellp] = P::from_f_raw(f[i]);
                *reinterpret_cast<float2*>(a.phi_dst + 2 * cellp) = mul2(phi, sp2(1.f / SC));
            }
            // every thread is done with the stages of rows y0 - 1 .. y0 + R - 2; ok becomes CTA-uniform
            ok = __syncthreads_and(ok) != 0;
            if (t == 0 && ok)
                for (int r = 0; r < TR; ++r)
                    if (j0 - 1 + r + TNS < nrow) issue(j0 - 1 + r + TNS);
        }
    }
    if (t == 0 && !ok) {
        // bounded wait for this CTA's copies still in flight before its shared memory is released
        for (unsigned q = issued > TNS ? issued - TNS : 0; q < issued; ++q)
            mbar_wait_bounded(bar0 + 8 * (q % TNS), (q / TNS) & 1u, nullptr, TMA_DRAIN_LIMIT);
    }
    (void)nxp;
}

// strips x planes x row ranges: the number of row ranges per (strip, plane)
// minimises the waves of resident CTAs times the rows one CTA stages (its range
// plus the two rows around it), so that the last wave is not left nearly empty
template <int STORE, int UK, bool WALLS, int R, int NS>
cudaError_t launch_tma_d3q15(const StepArgs& a, cudaStream_t st)
{
    constexpr int threads = T3_TP * R, smem = tma3_smem(NS);
    static int resident_by_dev[64] = {0};   // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    int& resident = resident_by_dev[dev & 63];
    if (resident == 0) {
        int nsm = 0, per_sm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step_tma_d3q15<STORE, UK, WALLS, R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_tma_d3q15<STORE, UK, WALLS, R, NS>, threads,
                                                      smem);
        resident = (nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
    }
    const int nstrip = a.nx / T3_W;
    long long nb = 1;
    double best = 1e300;
    for (long long b = 1; b <= 64 && b <= a.ny; ++b) {
        const long long ctas = (long long)nstrip * a.nz * b;
        const double waves = (double)((ctas + resident - 1) / resident);
        const double cost = waves * (double)((a.ny + b - 1) / b + 2);
        if (cost < best * 0.999) {
            best = cost;
            nb = b;
        }
    }
    k_step_tma_d3q15<STORE, UK, WALLS, R, NS>
        <<<dim3((unsigned)nstrip, (unsigned)a.nz, (unsigned)nb), threads, smem, st>>>(a, *a.tma15);
    return cudaGetLastError();
}

}  // namespace lbm
