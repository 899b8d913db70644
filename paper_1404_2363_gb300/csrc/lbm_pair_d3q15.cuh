// D3Q15 step for the 16-bit offset storage on node pairs: one thread owns the
// two adjacent nodes (x0, x0 + 1), x0 even, of one (y, z) row, and runs the
// decode, the collision (collide_d3q15<float2>) and the offset store for both
// with paired FP32 instructions. Offsets move as aligned 32-bit pairs, phi and
// the velocity factors as 64-bit pairs; a pull shifted by one column combines
// halves of two neighbouring pairs (offsets) or one pair and one scalar (phi,
// u). The FP16 form runs in units of 2^11 (its stored scale), as the D2Q9
// quad kernel does: the decode weights carry the factor, so no load or store
// multiplies.
//
// Decode of a pulled population from source s at step k:
//   f_i = g_i(s) + phi(s) (w_i + sum_d k_i e_id sched_d(k-1) a_d(s))
// with the schedule factor folded into the slopes (velocity fields), so a
// corner population costs three paired FMAs and an axis population one.
#pragma once
#include "lbm_pair.cuh"

namespace lbm {

// (v(x0 - e_x), v(x0 + 1 - e_x)) of one FP32 plane row; c = (v(x0), v(x0 + 1)),
// xlo = column x0 - 1, xhi = column x0 + 2 (periodic)
__device__ __forceinline__ float2 pair_window(const float* row, float2 c, int ex, int xlo, int xhi)
{
    if (ex == 0) return c;
    if (ex > 0) return make_float2(__ldg(row + xlo), c.x);
    return make_float2(c.y, __ldg(row + xhi));
}

// f^eq_i / phi = w_i + k_i e_i.u for two nodes with u given (wall rules)
__device__ __forceinline__ float2 feq_unit_pair15(float w0, float wa, float wd, float ka, float kd, int i,
                                                  float2 ux, float2 uy, float2 uz)
{
    using L = D3Q15;
    const int w = wclass<L>(i);
    if (w == 0) return sp2(w0);
    const float2 t[3] = {L::ex(i) > 0 ? ux : neg2(ux), L::ey(i) > 0 ? uy : neg2(uy), L::ez(i) > 0 ? uz : neg2(uz)};
    const bool on[3] = {L::ex(i) != 0, L::ey(i) != 0, L::ez(i) != 0};
    float2 eu = sp2(0.f);
    bool has = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (!on[d]) continue;
        eu = has ? add2(eu, t[d]) : t[d];
        has = true;
    }
    return w == 1 ? fma2(sp2(ka), eu, sp2(wa)) : fma2(sp2(kd), eu, sp2(wd));
}

// Needs nx even and 18 ncell < 2^31 (int offsets; checked by the launcher).
template <int STORE, int UK, bool WALLS>
__global__ void __launch_bounds__(256) k_step_pair_d3q15(const StepArgs a)
{
    using P = Pair<STORE>;
    using T2 = typename P::T2;
    using L = D3Q15;
    constexpr float SC = STORE == ST_F16 ? F16_SCALE : 1.f;   // working units (see above)
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int N = (int)a.ncell;
    const int y = blockIdx.y, z = blockIdx.z;
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= nx) return;
    const int xlo = x0 == 0 ? nx - 1 : x0 - 1;      // column x0 - 1
    const int xhi = x0 + 2 == nx ? 0 : x0 + 2;      // column x0 + 2
    const int xlp = x0 == 0 ? nx - 2 : x0 - 2;      // pair holding column x0 - 1
    // source rows by e_y + 1 and e_z + 1 (row y - e_y, plane z - e_z, periodic)
    const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
    const int zs[3] = {z + 1 == nz ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};
    const Coef& c = a.c;
    const T2* __restrict__ src = static_cast<const T2*>(a.src);   // pair index = cell / 2
    T2* __restrict__ dst = static_cast<T2*>(a.dst);
    const int NP = N / 2;
    float s_now[3], s_prev[3];
    sched_row_at(a.sched, a.srow_now, 3, s_now);
    sched_row_at(a.sched, a.srow_prev, 3, s_prev);
    const float w0 = c.w0 * SC, wa = c.wa * SC, wd = c.wd * SC;   // exact (power of two)
    const float ka = c.ka * SC, kd = c.kd * SC;
    float kas[3], kds[3];   // slopes with the schedule factor of u(k - 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        kas[d] = __fmul_rn(ka, s_prev[d]);
        kds[d] = __fmul_rn(kd, s_prev[d]);
    }

    // pull and decode
    float2 f[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const int row = (ys[ey + 1] + ny * zs[ez + 1]) * nx;   // first cell of the source row
        const T2* prow = src + (i * N + row) / 2;
        T2 h;
        if (ex == 0) h = ldg_pair(prow + x0 / 2);
        else if (ex > 0) h = P::join(ldg_pair(prow + xlp / 2), ldg_pair(prow + x0 / 2));
        else h = P::join(ldg_pair(prow + x0 / 2), ldg_pair(prow + xhi / 2));
        const float* prw = a.phi_src + row;
        const float2 ps = pair_window(prw, __ldg(reinterpret_cast<const float2*>(prw + x0)), ex, xlo, xhi);
        const int wc = wclass<L>(i);
        float2 e = sp2(wc == 0 ? w0 : (wc == 1 ? wa : wd));
        if (UK == U_FIELD) {
            const float* ks = wc == 1 ? kas : kds;
            const int ed[3] = {ex, ey, ez};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (ed[d] == 0) continue;
                const float* ar = a.ua + d * N + row;
                const float2 ad = pair_window(ar, __ldg(reinterpret_cast<const float2*>(ar + x0)), ex, xlo, xhi);
                e = fma2(sp2(ed[d] > 0 ? ks[d] : -ks[d]), ad, e);
            }
        } else if (UK == U_ROW && wc != 0) {
            const int yr = ys[ey + 1];
            const float ux = __fmul_rn(__ldg(a.ua + yr), s_prev[0]);
            const float uy = __fmul_rn(__ldg(a.ua + ny + yr), s_prev[1]);
            const float uz = __fmul_rn(__ldg(a.ua + 2 * ny + yr), s_prev[2]);
            e = sp2(fmaf(wc == 1 ? ka : kd, e_dot<L>(i, ux, uy, uz), wc == 1 ? wa : wd));
        }
        f[i] = fma2(ps, e, P::to_f_raw(h));
    }

    // own velocity factors a(x0), a(x0 + 1)
    const int cell = (y + ny * z) * nx + x0;
    const int cellp = cell / 2;
    float2 ao[3] = {sp2(0.f), sp2(0.f), sp2(0.f)};
    if (UK == U_FIELD) {
#pragma unroll
        for (int d = 0; d < 3; ++d) ao[d] = __ldg(reinterpret_cast<const float2*>(a.ua + d * N + cell));
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
                const float2 po = __ldg(reinterpret_cast<const float2*>(a.phi_src + cell));
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
    *reinterpret_cast<float2*>(a.phi_dst + cell) = mul2(phi, sp2(1.f / SC));
}

}  // namespace lbm
