// D3Q15 step for the 16-bit offset storage with its operands staged in shared
// memory along a walk in z (Appendix A lattice; arithmetic of k_step_pair_d3q15).
//
// A CTA of 32 TY threads owns a tile of 64 columns x TY rows (TY = 8 or 4) of
// the (x, y) plane and walks a range of z planes: warp w is row y0 + w of the
// tile, lane l the node pair (x0, x0 + 1) = (xt + 2 l, xt + 2 l + 1). Node
// (x, y, z) decodes population i from the offset g_i and from phi and the
// velocity factors a of its source (x - e_ix, y - e_iy, z - e_iz).
//
// Two kinds of shared-memory staging, both filled with 16-byte cp.async copies
// (each wrapped periodically on its own: nx is a multiple of 64, so no copy
// straddles the x edge) that hold no registers in flight:
//  - a ring of three plane slots with phi and a of the planes z - 1, z, z + 1
//    for the tile and a halo of 4 columns and 1 row on each side: each value
//    is fetched from L2 or HBM once per tile and read by its up to 15 pulls;
//  - the offsets one step pulls: for each population the TY source rows of
//    the tile (shifted by e_y, in plane z - e_z) over columns xt - 8 .. xt + 71.
// A step waits for its copies, decodes from shared memory, and after a
// barrier issues the copies of the next step (its offsets, and the plane
// z + 2 into the slot of plane z - 1) before its collision and stores, which
// the copies overlap. Pulls shifted in x join halves of two 32-bit offset
// pairs, as in k_step_pair_d3q15.
//
// The waits are the hardware's cp.async group waits and CTA barriers: no
// spin loop, so no wait limit applies.
#pragma once
#include "lbm_pair_d3q15.cuh"

namespace lbm {

constexpr int ZW_TX = 64;           // tile columns (32 node pairs: one warp)
constexpr int ZW_W = ZW_TX + 8;     // staged columns: xt - 4 .. xt + 67
constexpr int ZW_NS = 3;            // plane slots in the ring
constexpr int ZW_GW = ZW_TX + 16;   // staged offset columns: xt - 8 .. xt + 71

// Geometry of a tile of TY rows (TY warps per CTA, 4 or 8)
template <int TY>
struct ZwGeom {
    static constexpr int H = TY + 2;                    // staged rows: y0 - 1 .. y0 + TY
    static constexpr int PLANE = H * ZW_W;              // floats of one staged array of one plane
    static constexpr int CHUNKS = H * (ZW_W / 4);       // 16-byte copies per array and plane
    static constexpr int GPOS = TY * (ZW_GW / 8);       // 16-byte copies per population and step
    static_assert(CHUNKS <= 32 * TY, "one phi / a chunk per thread");
    static_assert(3 * GPOS <= 32 * TY, "three thread groups stage the offsets of five populations each");
};

__host__ __device__ constexpr int zw_arrays(int uk) { return uk == U_FIELD ? 4 : 1; }
__host__ __device__ constexpr int zw_smem(int uk, int ty)
{
    return ZW_NS * zw_arrays(uk) * (ty + 2) * ZW_W * 4 + 15 * ty * ZW_GW * 2;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// (v(x0 - e_x), v(x0 + 1 - e_x)) of a staged row; p points at column x0
__device__ __forceinline__ float2 zw_window(const float* p, int ex)
{
    const float2 c = *reinterpret_cast<const float2*>(p);
    if (ex == 0) return c;
    if (ex > 0) return make_float2(p[-1], c.x);
    return make_float2(c.y, p[2]);
}

// Offsets of populations P0 .. P0 + 4 (compile time) for step zs: this thread's
// position (row r, 16-byte column chunk q) of the tile's staged block of each,
// given as the rows y0 + r - e_y by e_y + 1 (yrow, times nx), the column xcol
// and the position sdst within a block.
template <int TY, int P0>
__device__ __forceinline__ void zw_issue_g(const uint16_t* __restrict__ g, uint16_t* gs, int N, int nxy, int nz,
                                           int zs, const int (&yrow)[3], int xcol, int sdst)
{
#pragma unroll
    for (int p = P0; p < P0 + 5; ++p) {
        const int ez = D3Q15::ez(p), ey = D3Q15::ey(p);
        int zp = zs - ez;
        zp = zp < 0 ? zp + nz : (zp >= nz ? zp - nz : zp);
        cp_async16(gs + p * (TY * ZW_GW) + sdst, g + p * N + zp * nxy + yrow[ey + 1] + xcol);
    }
}

// Needs nx % 64 == 0, ny % TY == 0, 18 ncell < 2^31 (int offsets) and 16-byte
// aligned offsets, phi and velocity fields (checked by the launcher).
// 80 registers: 3 CTAs of 256 threads (TY = 8) or 6 of 128 (TY = 4) per SM; at
// 64 registers, for a fourth 256-thread CTA, the kernel spills.
template <int STORE, int UK, bool WALLS, int TY>
__global__ void __launch_bounds__(32 * TY, TY == 8 ? 3 : 6) k_step_zw_d3q15(const StepArgs a)
{
    using Gm = ZwGeom<TY>;
    constexpr int PLANE = Gm::PLANE, CHUNKS = Gm::CHUNKS, GPOS = Gm::GPOS;
    using P = Pair<STORE>;
    using T2 = typename P::T2;
    using L = D3Q15;
    constexpr int NA = zw_arrays(UK);
    constexpr int SLOT = NA * PLANE;
    constexpr float SC = STORE == ST_F16 ? F16_SCALE : 1.f;   // working units (k_step_pair_d3q15)
    extern __shared__ __align__(16) float zs_m[];
    uint16_t* const gs = reinterpret_cast<uint16_t*>(zs_m + ZW_NS * SLOT);   // [15][TY][ZW_GW]
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int N = (int)a.ncell, NP = N / 2, nxy = nx * ny;
    const int t = threadIdx.x, lane = t & 31, ly = t >> 5;
    const int xt = (int)blockIdx.x * ZW_TX, y0 = (int)blockIdx.y * TY;
    const int x0 = xt + 2 * lane, y = y0 + ly;
    const int zb = (int)((long long)blockIdx.z * nz / gridDim.z);
    const int ze = (int)((long long)(blockIdx.z + 1) * nz / gridDim.z);
    if (zb >= ze) return;
    const int nplanes = ze - zb + 2;   // staged planes zb - 1 .. ze (periodic)

    // phi / a fill: thread t < CHUNKS copies the 16 bytes at staged row
    // t / (ZW_W / 4), columns 4 (t % (ZW_W / 4)) .. + 3, of every staged array;
    // fixed for the walk, so per plane only the plane offset changes
    int fsrc = 0, fdst = 0;
    if (t < CHUNKS) {
        const int r = t / (ZW_W / 4), q = t - r * (ZW_W / 4);
        int yy = y0 - 1 + r;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        int xx = xt - 4 + 4 * q;
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        fsrc = yy * nx + xx;
        fdst = r * ZW_W + 4 * q;
    }
    auto issue_plane = [&](int j) {   // plane zb - 1 + j into slot j % ZW_NS
        if (j < nplanes && t < CHUNKS) {
            int zp = zb - 1 + j;
            zp = zp < 0 ? zp + nz : (zp >= nz ? zp - nz : zp);
            float* sd = zs_m + (j % ZW_NS) * SLOT + fdst;
            const int go = zp * nxy + fsrc;
            cp_async16(sd, a.phi_src + go);
            if (UK == U_FIELD) {
#pragma unroll
                for (int d = 0; d < 3; ++d) cp_async16(sd + (1 + d) * PLANE, a.ua + d * N + go);
            }
        }
    };
    // offset fill: thread t < 3 GPOS stages position t % GPOS (row r, chunk q)
    // of populations 5 (t / GPOS) .. + 4
    const int gpos = t % GPOS, ggrp = t / GPOS;
    int gyrow[3], gxcol, gsdst;
    {
        const int r = gpos / (ZW_GW / 8), q = gpos - r * (ZW_GW / 8);
#pragma unroll
        for (int k = 0; k < 3; ++k) {   // rows y0 + r - e_y by e_y + 1 = k
            int yy = y0 + r + 1 - k;
            yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            gyrow[k] = yy * nx;
        }
        int xx = xt - 8 + 8 * q;
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        gxcol = xx;
        gsdst = r * ZW_GW + 8 * q;
    }
    const uint16_t* const g16 = static_cast<const uint16_t*>(a.src);
    auto issue_g = [&](int zs) {   // offsets pulled by step zs
        if (zs < ze) {
            if (ggrp == 0) zw_issue_g<TY, 0>(g16, gs, N, nxy, nz, zs, gyrow, gxcol, gsdst);
            else if (ggrp == 1) zw_issue_g<TY, 5>(g16, gs, N, nxy, nz, zs, gyrow, gxcol, gsdst);
            else if (ggrp == 2) zw_issue_g<TY, 10>(g16, gs, N, nxy, nz, zs, gyrow, gxcol, gsdst);
        }
    };

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
    const int yr3[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};   // row y - e_y by e_y + 1
    const int own = (1 + ly) * ZW_W + 4 + 2 * lane;   // the pair's staged position in a plane slot
    // the pair's offsets in the staged block of a population: 32-bit words at
    // columns x0 - 2, x0, x0 + 2 of row ly (block column xt - 8 + j is j)
    const unsigned* const gw = reinterpret_cast<const unsigned*>(gs) + (ly * ZW_GW + 8 + 2 * lane) / 2;

    // one copy group per step: the prologue stages planes 0 .. 2 and the offsets of
    // step zb; step r, once its decode is done, stages plane r + 3 (into the slot of
    // plane r) and the offsets of step zb + r + 1, which its collision and stores
    // then overlap
#pragma unroll 1
    for (int j = 0; j < ZW_NS; ++j) issue_plane(j);
    issue_g(zb);
    cp_async_commit();

#pragma unroll 1
    for (int r = 0; r < ze - zb; ++r) {
        const int z = zb + r;
        cp_async_wait<0>();   // planes z - 1 .. z + 1 and the offsets of step z have landed
        __syncthreads();
        // slot of plane z - e_z by e_z + 1: z + 1, z, z - 1 (walk indices r + 2, r + 1, r)
        const float* S[3] = {zs_m + ((r + 2) % ZW_NS) * SLOT + own, zs_m + ((r + 1) % ZW_NS) * SLOT + own,
                             zs_m + (r % ZW_NS) * SLOT + own};

        // pull and decode
        float2 f[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) {
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            const unsigned* w = gw + i * (TY * ZW_GW / 2);
            unsigned hw;
            if (ex == 0) hw = w[0];
            else if (ex > 0) hw = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(w[-1]), QuadH<STORE>::as_t2(w[0])));
            else hw = QuadH<STORE>::as_u(P::join(QuadH<STORE>::as_t2(w[0]), QuadH<STORE>::as_t2(w[1])));
            const float* sp = S[ez + 1] - ey * ZW_W;   // source row in the slot, column x0
            const float2 ps = zw_window(sp, ex);
            const int wc = wclass<L>(i);
            float2 e = sp2(wc == 0 ? w0 : (wc == 1 ? wa : wd));
            if (UK == U_FIELD) {
                const float* ks = wc == 1 ? kas : kds;
                const int ed[3] = {ex, ey, ez};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (ed[d] == 0) continue;
                    const float2 ad = zw_window(sp + (1 + d) * PLANE, ex);
                    e = fma2(sp2(ed[d] > 0 ? ks[d] : -ks[d]), ad, e);
                }
            } else if (UK == U_ROW && wc != 0) {
                const int yr = yr3[ey + 1];
                const float ux = __fmul_rn(__ldg(a.ua + yr), s_prev[0]);
                const float uy = __fmul_rn(__ldg(a.ua + ny + yr), s_prev[1]);
                const float uz = __fmul_rn(__ldg(a.ua + 2 * ny + yr), s_prev[2]);
                e = sp2(fmaf(wc == 1 ? ka : kd, e_dot<L>(i, ux, uy, uz), wc == 1 ? wa : wd));
            }
            f[i] = fma2(ps, e, P::to_f_raw(QuadH<STORE>::as_t2(hw)));
        }
        // own velocity factors a(x0), a(x0 + 1) and phi (plane z: not refilled below)
        float2 ao[3] = {sp2(0.f), sp2(0.f), sp2(0.f)};
        if (UK == U_FIELD) {
#pragma unroll
            for (int d = 0; d < 3; ++d) ao[d] = *reinterpret_cast<const float2*>(S[1] + (1 + d) * PLANE);
        } else if (UK == U_ROW) {
#pragma unroll
            for (int d = 0; d < 3; ++d) ao[d] = sp2(__ldg(a.ua + d * ny + y));
        }
        const float2 po = *reinterpret_cast<const float2*>(S[1]);

        __syncthreads();   // the offsets of step z and the slot of plane z - 1 are free
        issue_plane(r + ZW_NS);
        issue_g(z + 1);
        cp_async_commit();

        const int cellp = (z * nxy + y * nx + x0) >> 1;   // the pair's own index
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
        reinterpret_cast<float2*>(a.phi_dst)[cellp] = mul2(phi, sp2(1.f / SC));
    }
    cp_async_wait<0>();   // no copy outlives the CTA's shared memory
}

// tiles x z ranges: the number of z ranges per tile minimises the waves of
// resident CTAs times the planes one CTA stages (its range plus the two planes
// around it), so that the last wave is not left nearly empty; a walk length set
// by lbm_cde_set_zwalk is kept instead
template <int STORE, int UK, bool WALLS, int TY>
cudaError_t launch_zw_d3q15(const StepArgs& a, cudaStream_t st)
{
    constexpr int threads = 32 * TY, smem = zw_smem(UK, TY);
    static int resident_by_dev[64] = {0};   // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    int& resident = resident_by_dev[dev & 63];
    if (resident == 0) {
        int nsm = 0, per_sm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step_zw_d3q15<STORE, UK, WALLS, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_zw_d3q15<STORE, UK, WALLS, TY>, threads, smem);
        resident = (nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
    }
    const long long tiles = (long long)(a.nx / ZW_TX) * (a.ny / TY);
    long long nb = a.zwalk > 0 ? (a.nz + a.zwalk - 1) / a.zwalk : 1;
    if (a.zwalk <= 0) {
        double best = 1e300;
        for (long long b = 1; b <= 64 && b <= a.nz; ++b) {
            const long long ctas = tiles * b;
            const double waves = (double)((ctas + resident - 1) / resident);
            const double cost = waves * (double)((a.nz + b - 1) / b + 2);
            if (cost < best * 0.999) {
                best = cost;
                nb = b;
            }
        }
    }
    k_step_zw_d3q15<STORE, UK, WALLS, TY>
        <<<dim3((unsigned)(a.nx / ZW_TX), (unsigned)(a.ny / TY), (unsigned)nb), threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lbm
