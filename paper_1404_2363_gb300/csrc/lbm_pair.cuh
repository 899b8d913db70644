// D2Q9 step for the 16-bit offset storage on node pairs: one thread owns the
// two adjacent nodes (x0, x0 + 1), x0 even, and evaluates the decode, the
// collision and the offset store for both with paired FP32 instructions
// (add/mul/fma on float2, sm_100 and later), so every arithmetic instruction
// serves two nodes. The offsets are loaded as aligned 32-bit pairs; the
// pulls shifted by one column combine halves of two neighbouring pairs.
//
// The operation sequence is the one of collide<D2Q9, true> and of the decode
// in k_step; the compiler may fuse some paired multiplies into the adds that
// follow them, so results agree with k_step to FP32 rounding.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

// Paired operations (one instruction for both nodes). The compiler may fuse a
// paired multiply into a following paired add, so the pair kernel agrees with
// the one-node kernel to FP32 rounding rather than bit for bit.
__device__ __forceinline__ float2 sp2(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// collide<D2Q9, true> for two nodes: the offsets g = M^-1 (m' - m^eq) of the
// 16-bit forms, whose equilibria are linear in u (see lbm_device.cuh)
__device__ __forceinline__ float2 collide_pair(float2 (&v)[9], float2 ux, float2 uy, const Coef& c)
{
    // m = M v by same-speed sums and differences
    const float2 sx = add2(v[1], v[3]), ax = sub2(v[1], v[3]);
    const float2 sy = add2(v[2], v[4]), ay = sub2(v[2], v[4]);
    const float2 p57 = add2(v[5], v[7]), d57 = sub2(v[5], v[7]);
    const float2 p68 = add2(v[6], v[8]), d68 = sub2(v[6], v[8]);
    const float2 sa = add2(sx, sy), sd = add2(p57, p68);
    const float2 jx = sub2(d57, d68), jy = add2(d57, d68);
    const float2 phi = add2(add2(v[0], sa), sd);
    const float2 m1 = fma2(sp2(2.f), sd, fma2(sp2(-4.f), v[0], neg2(sa)));
    const float2 m2 = fma2(sp2(-2.f), sa, fma2(sp2(4.f), v[0], sd));
    const float2 m3 = add2(ax, jx), m4 = fma2(sp2(-2.f), ax, jx);
    const float2 m5 = add2(ay, jy), m6 = fma2(sp2(-2.f), ay, jy);
    const float2 m7 = sub2(sx, sy), m8 = sub2(p57, p68);
    // dl = m - m^eq; a = diag(1/|M_k|^2) (I - S) dl with the folded c.ro, c.fr
    const float2 dl1 = fma2(sp2(-c.meq1), phi, m1), dl2 = fma2(sp2(-c.meq2), phi, m2);
    const float2 dl3 = fma2(neg2(phi), ux, m3), dl4 = fma2(phi, ux, m4);
    const float2 dl5 = fma2(neg2(phi), uy, m5), dl6 = fma2(phi, uy, m6);
    const float2 a1 = mul2(dl1, sp2(c.ro[1])), a2 = mul2(dl2, sp2(c.ro[2]));
    const float2 a4 = mul2(dl4, sp2(c.ro[4])), a6 = mul2(dl6, sp2(c.ro[6]));
    const float2 a7 = mul2(m7, sp2(c.ro[7])), a8 = mul2(m8, sp2(c.ro[8]));
    const float2 a3 = fma2(sp2(c.fr[0]), dl3, fma2(sp2(c.fr[1]), dl4, fma2(sp2(c.fr[2]), dl5, mul2(sp2(c.fr[3]), dl6))));
    const float2 a5 = fma2(sp2(c.fr[4]), dl3, fma2(sp2(c.fr[5]), dl4, fma2(sp2(c.fr[6]), dl5, mul2(sp2(c.fr[7]), dl6))));
    // v = M^T a (populations<D2Q9, true, false>)
    const float2 A = fma2(sp2(-2.f), a2, neg2(a1));
    const float2 B = fma2(sp2(2.f), a1, a2);
    const float2 X = fma2(sp2(-2.f), a4, a3), Y = fma2(sp2(-2.f), a6, a5);
    const float2 Xd = add2(a3, a4), Yd = add2(a5, a6);
    const float2 AP = add2(A, a7), AM = sub2(A, a7);
    const float2 BP = add2(B, a8), BM = sub2(B, a8);
    const float2 XY = add2(Xd, Yd), XmY = sub2(Xd, Yd);
    v[1] = add2(AP, X);
    v[3] = sub2(AP, X);
    v[2] = add2(AM, Y);
    v[4] = sub2(AM, Y);
    v[5] = add2(BP, XY);
    v[7] = sub2(BP, XY);
    v[6] = sub2(BM, XmY);
    v[8] = add2(BM, XmY);
    v[0] = fma2(sp2(-c.eps0), phi, neg2(mul2(sp2(4.f), add2(A, B))));   // 4 x exact; Coef::eps0
    return phi;
}

// collide<D2Q9, false> for two nodes: post-collision populations, with the
// u^2 terms of MRT-B1/B2. CC is any constants type with the fields collide reads.
template <class CC>
__device__ __forceinline__ float2 collide_pair_f32(float2 (&v)[9], float2 ux, float2 uy, const CC& c)
{
    const float2 sx = add2(v[1], v[3]), ax = sub2(v[1], v[3]);
    const float2 sy = add2(v[2], v[4]), ay = sub2(v[2], v[4]);
    const float2 p57 = add2(v[5], v[7]), d57 = sub2(v[5], v[7]);
    const float2 p68 = add2(v[6], v[8]), d68 = sub2(v[6], v[8]);
    const float2 sa = add2(sx, sy), sd = add2(p57, p68);
    const float2 jx = sub2(d57, d68), jy = add2(d57, d68);
    const float2 phi = add2(add2(v[0], sa), sd);
    const float2 m1 = fma2(sp2(2.f), sd, fma2(sp2(-4.f), v[0], neg2(sa)));
    const float2 m2 = fma2(sp2(-2.f), sa, fma2(sp2(4.f), v[0], sd));
    const float2 m3 = add2(ax, jx), m4 = fma2(sp2(-2.f), ax, jx);
    const float2 m5 = add2(ay, jy), m6 = fma2(sp2(-2.f), ay, jy);
    const float2 m7 = sub2(sx, sy), m8 = sub2(p57, p68);
    // d = m - m^eq (Eq. 15 with the MRT-B1/B2 u^2 terms when present)
    float2 d1 = fma2(sp2(-c.meq1), phi, m1), d2 = fma2(sp2(-c.meq2), phi, m2);
    const float2 d3 = fma2(neg2(phi), ux, m3), d4 = fma2(phi, ux, m4);
    const float2 d5 = fma2(neg2(phi), uy, m5), d6 = fma2(phi, uy, m6);
    float2 d7 = m7, d8 = m8;
    if (c.b1 != 0.f || c.b2 != 0.f || c.g7 != 0.f || c.g8 != 0.f) {
        const float2 uyy = mul2(uy, uy);
        const float2 u2 = fma2(ux, ux, uyy);
        d1 = fma2(mul2(sp2(-c.b1), u2), phi, d1);
        d2 = fma2(mul2(sp2(-c.b2), u2), phi, d2);
        d7 = fma2(mul2(sp2(-c.g7), fma2(ux, ux, neg2(uyy))), phi, d7);
        d8 = fma2(mul2(sp2(-c.g8), mul2(ux, uy)), phi, d8);
    }
    // m' = m - S d (Eq. 31), scaled by 1/|M_k|^2
    float2 r0 = fma2(sp2(c.A[0]), d3, sp2(0.f));
    r0 = fma2(sp2(c.C[0]), d4, r0);
    r0 = fma2(sp2(c.A[1]), d5, r0);
    r0 = fma2(sp2(c.C[1]), d6, r0);
    float2 r1 = fma2(sp2(c.A[2]), d3, sp2(0.f));
    r1 = fma2(sp2(c.C[2]), d4, r1);
    r1 = fma2(sp2(c.A[3]), d5, r1);
    r1 = fma2(sp2(c.C[3]), d6, r1);
    const float2 a0 = mul2(phi, sp2(1.f / 9.f));
    const float2 a1 = mul2(fma2(sp2(-c.s[1]), d1, m1), sp2(1.f / 36.f));
    const float2 a2 = mul2(fma2(sp2(-c.s[2]), d2, m2), sp2(1.f / 36.f));
    const float2 a3 = mul2(sub2(m3, r0), sp2(1.f / 6.f));
    const float2 a4 = mul2(fma2(sp2(-c.s[4]), d4, m4), sp2(1.f / 12.f));
    const float2 a5 = mul2(sub2(m5, r1), sp2(1.f / 6.f));
    const float2 a6 = mul2(fma2(sp2(-c.s[6]), d6, m6), sp2(1.f / 12.f));
    const float2 a7 = mul2(fma2(sp2(-c.s[7]), d7, m7), sp2(0.25f));
    const float2 a8 = mul2(fma2(sp2(-c.s[8]), d8, m8), sp2(0.25f));
    // f' = M^T a (populations<D2Q9, false, false>), rest population from the mass balance
    const float2 A = fma2(sp2(-2.f), a2, sub2(a0, a1));
    const float2 B = fma2(sp2(2.f), a1, add2(a0, a2));
    const float2 X = fma2(sp2(-2.f), a4, a3), Y = fma2(sp2(-2.f), a6, a5);
    const float2 Xd = add2(a3, a4), Yd = add2(a5, a6);
    const float2 AP = add2(A, a7), AM = sub2(A, a7);
    const float2 BP = add2(B, a8), BM = sub2(B, a8);
    const float2 XY = add2(Xd, Yd), XmY = sub2(Xd, Yd);
    v[1] = add2(AP, X);
    v[3] = sub2(AP, X);
    v[2] = add2(AM, Y);
    v[4] = sub2(AM, Y);
    v[5] = add2(BP, XY);
    v[7] = sub2(BP, XY);
    v[6] = sub2(BM, XmY);
    v[8] = add2(BM, XmY);
    v[0] = sub2(phi, mul2(sp2(4.f), add2(A, B)));
    return phi;
}

// paired 16-bit words
template <int S> struct Pair;
template <> struct Pair<ST_F16> {
    using T2 = __half2;
    static constexpr float scale = F16_SCALE;   // stored value = scale x offset
    __device__ static float2 to_f(__half2 h) { return mul2(__half22float2(h), sp2(1.0f / F16_SCALE)); }
    __device__ static __half2 from_f(float2 v) { return __float22half2_rn(mul2(v, sp2(F16_SCALE))); }
    __device__ static float2 to_f_raw(__half2 h) { return __half22float2(h); }
    __device__ static __half2 from_f_raw(float2 v) { return __float22half2_rn(v); }
    __device__ static __half2 join(__half2 lo_src, __half2 hi_src) {   // (lo_src.y, hi_src.x)
        return __halves2half2(__high2half(lo_src), __low2half(hi_src));
    }
};
template <> struct Pair<ST_BF16> {
    using T2 = __nv_bfloat162;
    static constexpr float scale = 1.f;
    __device__ static float2 to_f(__nv_bfloat162 h) { return __bfloat1622float2(h); }
    __device__ static __nv_bfloat162 from_f(float2 v) { return __float22bfloat162_rn(v); }
    __device__ static float2 to_f_raw(__nv_bfloat162 h) { return __bfloat1622float2(h); }
    __device__ static __nv_bfloat162 from_f_raw(float2 v) { return __float22bfloat162_rn(v); }
    __device__ static __nv_bfloat162 join(__nv_bfloat162 lo_src, __nv_bfloat162 hi_src) {
        return __halves2bfloat162(__high2bfloat16(lo_src), __low2bfloat16(hi_src));
    }
};

template <class T2>
__device__ __forceinline__ T2 ldg_pair(const T2* p)
{
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<const T2*>(&w);
}

// f^eq_i / phi = w_i + k_i e_i.u for two nodes (feq_unit<D2Q9>)
__device__ __forceinline__ float2 feq_unit_pair(const Coef& c, int i, float2 ux, float2 uy)
{
    const int w = wclass<D2Q9>(i);
    if (w == 0) return sp2(c.w0);
    const int ex = D2Q9::ex(i), ey = D2Q9::ey(i);
    float2 eu;
    if (ey == 0) eu = ex > 0 ? ux : neg2(ux);
    else if (ex == 0) eu = ey > 0 ? uy : neg2(uy);
    else if (ex > 0) eu = ey > 0 ? add2(ux, uy) : sub2(ux, uy);
    else eu = ey > 0 ? sub2(uy, ux) : neg2(add2(ux, uy));
    return w == 1 ? fma2(sp2(c.ka), eu, sp2(c.wa)) : fma2(sp2(c.kd), eu, sp2(c.wd));
}

// Needs nx even and 12 ncell < 2^31 (int offsets; checked by the launcher).
template <int STORE, int UK, bool WALLS>
__global__ void __launch_bounds__(256) k_step_pair_d2q9(const StepArgs a)
{
    using P = Pair<STORE>;
    using T2 = typename P::T2;
    using L = D2Q9;
    const int nx = a.nx, ny = a.ny;
    const int N = (int)a.ncell;
    const int y = blockIdx.y;
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= nx) return;
    const int xl = x0 == 0 ? nx - 2 : x0 - 2;       // pair holding column x0 - 1
    const int xr = x0 + 2 == nx ? 0 : x0 + 2;       // pair holding column x0 + 2
    const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};   // source row by e_y + 1
    const Coef& c = a.c;
    const T2* __restrict__ src = static_cast<const T2*>(a.src);   // pair index = cell / 2
    T2* __restrict__ dst = static_cast<T2*>(a.dst);
    const int NP = N / 2, nxp = nx / 2;
    float s_now[3], s_prev[3];
    sched_row_at(a.sched, a.srow_now, 2, s_now);
    sched_row_at(a.sched, a.srow_prev, 2, s_prev);

    // phi and u(k-1) at the sources: for source row r (by e_y + 1) the column
    // pairs (x0 - 1, x0), (x0, x0 + 1), (x0 + 1, x0 + 2) (by 1 - e_x)
    float2 Ps[3][3], Ux[3][3], Uy[3][3];
    float2 axo = sp2(0.f), ayo = sp2(0.f);   // own raw velocity factors a(x0), a(x0 + 1)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int row = ys[r] * nx;
        const float2 pm = __ldg(reinterpret_cast<const float2*>(a.phi_src + row + x0));
        const float pl = __ldg(a.phi_src + row + xl + 1), pr = __ldg(a.phi_src + row + xr);
        Ps[r][0] = make_float2(pl, pm.x);
        Ps[r][1] = pm;
        Ps[r][2] = make_float2(pm.y, pr);
        if (UK == U_FIELD) {
            const float* ax = a.ua;
            const float* ay = a.ua + a.ncell;
            const float2 xm = __ldg(reinterpret_cast<const float2*>(ax + row + x0));
            const float xlv = __ldg(ax + row + xl + 1), xrv = __ldg(ax + row + xr);
            const float2 ym = __ldg(reinterpret_cast<const float2*>(ay + row + x0));
            const float ylv = __ldg(ay + row + xl + 1), yrv = __ldg(ay + row + xr);
            Ux[r][0] = mul2(make_float2(xlv, xm.x), sp2(s_prev[0]));
            Ux[r][1] = mul2(xm, sp2(s_prev[0]));
            Ux[r][2] = mul2(make_float2(xm.y, xrv), sp2(s_prev[0]));
            Uy[r][0] = mul2(make_float2(ylv, ym.x), sp2(s_prev[1]));
            Uy[r][1] = mul2(ym, sp2(s_prev[1]));
            Uy[r][2] = mul2(make_float2(ym.y, yrv), sp2(s_prev[1]));
            if (r == 1) {
                axo = xm;
                ayo = ym;
            }
        } else if (UK == U_ROW) {
            const float ux = __fmul_rn(__ldg(a.ua + ys[r]), s_prev[0]);
            const float uy = __fmul_rn(__ldg(a.ua + a.ny + ys[r]), s_prev[1]);
            Ux[r][0] = Ux[r][1] = Ux[r][2] = sp2(ux);
            Uy[r][0] = Uy[r][1] = Uy[r][2] = sp2(uy);
            if (r == 1) {
                axo = sp2(__ldg(a.ua + y));
                ayo = sp2(__ldg(a.ua + a.ny + y));
            }
        } else {
            Ux[r][0] = Ux[r][1] = Ux[r][2] = sp2(0.f);
            Uy[r][0] = Uy[r][1] = Uy[r][2] = sp2(0.f);
        }
    }

    // pull and decode f_i = g_i(s) + phi(s) f^eq_i(1, u(s, k-1))
    float2 f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ex = L::ex(i), ey = L::ey(i);
        const int r = ey + 1, cp = 1 - ex;
        const T2* row = src + i * NP + ys[r] * nxp;
        T2 h;
        if (ex == 0) h = ldg_pair(row + x0 / 2);
        else if (ex > 0) h = P::join(ldg_pair(row + xl / 2), ldg_pair(row + x0 / 2));
        else h = P::join(ldg_pair(row + x0 / 2), ldg_pair(row + xr / 2));
        f[i] = fma2(Ps[r][cp], feq_unit_pair(c, i, Ux[r][cp], Uy[r][cp]), P::to_f(h));
    }
    const int cellp = y * nxp + x0 / 2;
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
                        const float2 g = P::to_f(ldg_pair(src + o * NP + cellp));
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


// ---------------------------------------------------------------------------
// D2Q9 step on node quads: one thread owns x0 .. x0 + 3 (x0 = 4 t, nx % 4 == 0)
// of one row and moves its data with 128-bit (FP32) or 64-bit (16-bit)
// loads and stores. A pull shifted by one column needs one element of the
// neighbouring quad: it comes from the adjacent lane by a warp shuffle, and
// from memory only at warp edges and at the periodic seam. The decode is
// scalar; the collisions run as two paired FP32 pairs (collide_pair /
// collide_pair_f32). The FP16 form runs in units of 2^11 (the stored scale):
// the decode weights are scaled by 2^11, so the pulled populations, the
// collision and the new offsets all carry the factor exactly (a power of two)
// and neither the loads nor the stores multiply; only phi is scaled back.
// ---------------------------------------------------------------------------
template <int STORE> struct Quad;
template <> struct Quad<ST_F32> {
    // quad of plane values at columns x0 .. x0 + 3
    using W = float4;
    __device__ static W load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
};

template <int STORE>
struct QuadH {   // 16-bit: two 32-bit words (x0, x0 + 1), (x0 + 2, x0 + 3)
    using T2 = typename Pair<STORE>::T2;
    __device__ static uint2 load(const void* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
    __device__ static T2 as_t2(unsigned w) { return *reinterpret_cast<const T2*>(&w); }
    __device__ static unsigned as_u(T2 h) { return *reinterpret_cast<const unsigned*>(&h); }
};

// The six window values v(x0 - 1) .. v(x0 + 4) of one FP32 plane row around the quad.
__device__ __forceinline__ void window6(const float* row, int x0c, int xl, int xr, bool needL, bool needR,
                                        float (&w)[6])
{
    const float4 m = __ldg(reinterpret_cast<const float4*>(row + x0c));
    float l = __shfl_up_sync(0xffffffffu, m.w, 1);
    float r = __shfl_down_sync(0xffffffffu, m.x, 1);
    if (needL) l = __ldg(row + xl);
    if (needR) r = __ldg(row + xr);
    w[0] = l;
    w[1] = m.x;
    w[2] = m.y;
    w[3] = m.z;
    w[4] = m.w;
    w[5] = r;
}

template <int STORE, int UK, bool WALLS>
__global__ void __launch_bounds__(256, 4) k_step_quad_d2q9(const StepArgs a)
{
    using L = D2Q9;
    constexpr bool NEQ = STORE != ST_F32;
    constexpr float SC = STORE == ST_F16 ? F16_SCALE : 1.f;   // working units (see above)
    const int nx = a.nx, ny = a.ny;
    const int N = (int)a.ncell;
    const int y = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int x0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool live = x0 < nx;
    const int x0c = live ? x0 : nx - 4;             // dead lanes still take part in the shuffles
    const int xl = x0c == 0 ? nx - 1 : x0c - 1;     // column x0 - 1
    const int xr = x0c + 4 == nx ? 0 : x0c + 4;     // column x0 + 4
    const bool needL = lane == 0 || x0c == 0;
    const bool needR = lane == 31 || x0c + 4 >= nx;
    const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};   // source row by e_y + 1
    const Coef& c = a.c;
    Coef cd = a.c;    // decode weights in working units
    if (SC != 1.f) {
        cd.w0 *= SC;
        cd.wa *= SC;
        cd.wd *= SC;
        cd.ka *= SC;
        cd.kd *= SC;
    }
    float s_now[3], s_prev[3];
    sched_row_at(a.sched, a.srow_now, 2, s_now);
    sched_row_at(a.sched, a.srow_prev, 2, s_prev);

    float f[9][4];    // pulled (and decoded) populations of the four nodes, working units
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int row = ys[r] * nx;
        float P[6], Ux[6], Uy[6];
        if (NEQ) {
            window6(a.phi_src + row, x0c, xl, xr, needL, needR, P);
            if (UK == U_FIELD) {
                window6(a.ua + row, x0c, xl, xr, needL, needR, Ux);
                window6(a.ua + N + row, x0c, xl, xr, needL, needR, Uy);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    Ux[k] = __fmul_rn(Ux[k], s_prev[0]);
                    Uy[k] = __fmul_rn(Uy[k], s_prev[1]);
                }
            } else {
                float ux = 0.f, uy = 0.f;
                if (UK == U_ROW) {
                    ux = __fmul_rn(__ldg(a.ua + ys[r]), s_prev[0]);
                    uy = __fmul_rn(__ldg(a.ua + a.ny + ys[r]), s_prev[1]);
                }
#pragma unroll
                for (int k = 0; k < 6; ++k) Ux[k] = ux, Uy[k] = uy;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (L::ey(i) + 1 != r) continue;
            const int ex = L::ex(i);
            float g[4];
            if constexpr (!NEQ) {
                float w[6];
                const float* prow = static_cast<const float*>(a.src) + i * N + row;
                if (ex == 0) {
                    const float4 m = __ldg(reinterpret_cast<const float4*>(prow + x0c));
                    g[0] = m.x, g[1] = m.y, g[2] = m.z, g[3] = m.w;
                } else {
                    window6(prow, x0c, xl, xr, needL && ex > 0, needR && ex < 0, w);
#pragma unroll
                    for (int j = 0; j < 4; ++j) g[j] = w[j + 1 - ex];
                }
            } else {
                using Q = QuadH<STORE>;
                using P2 = Pair<STORE>;
                const unsigned short* prow = static_cast<const unsigned short*>(a.src) + i * N + row;
                const uint2 m = Q::load(prow + x0c);
                unsigned w0 = m.x, w1 = m.y;
                if (ex > 0) {            // columns x0 - 1 .. x0 + 2
                    unsigned lw = __shfl_up_sync(0xffffffffu, m.y, 1);
                    if (needL) lw = __ldg(reinterpret_cast<const unsigned*>(prow + (x0c == 0 ? nx - 2 : x0c - 2)));
                    w0 = Q::as_u(P2::join(Q::as_t2(lw), Q::as_t2(m.x)));
                    w1 = Q::as_u(P2::join(Q::as_t2(m.x), Q::as_t2(m.y)));
                } else if (ex < 0) {     // columns x0 + 1 .. x0 + 4
                    unsigned rw = __shfl_down_sync(0xffffffffu, m.x, 1);
                    if (needR) rw = __ldg(reinterpret_cast<const unsigned*>(prow + xr));
                    w0 = Q::as_u(P2::join(Q::as_t2(m.x), Q::as_t2(m.y)));
                    w1 = Q::as_u(P2::join(Q::as_t2(m.y), Q::as_t2(rw)));
                }
                const float2 g01 = P2::to_f_raw(Q::as_t2(w0)), g23 = P2::to_f_raw(Q::as_t2(w1));
                g[0] = g01.x, g[1] = g01.y, g[2] = g23.x, g[3] = g23.y;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float v = g[j];
                if (NEQ) {
                    const int sidx = j + 1 - ex;     // source column x0 + j - e_x in the window
                    v = fmaf(P[sidx], feq_unit<L>(cd, i, Ux[sidx], Uy[sidx], 0.f), v);
                }
                f[i][j] = v;
            }
        }
    }

    // own raw velocity factors (for u(k) and the walls)
    float axo[4] = {0.f, 0.f, 0.f, 0.f}, ayo[4] = {0.f, 0.f, 0.f, 0.f};
    if (UK == U_FIELD) {
        const float4 ax = __ldg(reinterpret_cast<const float4*>(a.ua + y * nx + x0c));
        const float4 ay = __ldg(reinterpret_cast<const float4*>(a.ua + N + y * nx + x0c));
        axo[0] = ax.x, axo[1] = ax.y, axo[2] = ax.z, axo[3] = ax.w;
        ayo[0] = ay.x, ayo[1] = ay.y, ayo[2] = ay.z, ayo[3] = ay.w;
    } else if (UK == U_ROW) {
        const float ax = __ldg(a.ua + y), ay = __ldg(a.ua + a.ny + y);
#pragma unroll
        for (int j = 0; j < 4; ++j) axo[j] = ax, ayo[j] = ay;
    }
    const int cell = y * nx + x0c;
    if (WALLS) {
        const bool lo = (y == 0) && a.bc_lo != BC_PERIODIC;
        const bool hi = (y == ny - 1) && a.bc_hi != BC_PERIODIC;
        if (lo || hi) {
            const int kind = lo ? a.bc_lo : a.bc_hi;
            const int inward = lo ? 1 : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float ux = UK == U_NONE ? 0.f : __fmul_rn(axo[j], s_prev[0]);
                const float uy = UK == U_NONE ? 0.f : __fmul_rn(ayo[j], s_prev[1]);
                if (kind == BC_NOFLUX) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (L::ey(i) == inward) f[i][j] = f[mirror_y<L>(i)][j];
                } else if (kind == BC_BOUNCE) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (L::ey(i) == inward) {
                            const int o = opposite<L>(i);
                            using T = typename StT<STORE>::T;
                            float v = ldg_f(static_cast<const T*>(a.src) + o * N + cell + j) * SC;   // exact
                            if (NEQ) v = fmaf(__ldg(a.phi_src + cell + j), feq_unit<L>(cd, o, ux, uy, 0.f), v);
                            f[i][j] = v;
                        }
                } else {   // Dirichlet
                    float known = 0.f, wk = 0.f;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (L::ey(i) == inward) wk += feq_unit<L>(cd, i, ux, uy, 0.f);
                        else known += f[i][j];
                    }
                    const float ps = ((lo ? a.phiw_lo : a.phiw_hi) * SC - known) / wk;
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (L::ey(i) == inward) f[i][j] = __fmul_rn(ps, feq_unit<L>(cd, i, ux, uy, 0.f));
                }
            }
        }
    }
    // collisions of the pairs (x0, x0 + 1) and (x0 + 2, x0 + 3)
    float2 out[2][9], phi[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = make_float2(f[i][2 * h], f[i][2 * h + 1]);
        float2 ux = sp2(0.f), uy = sp2(0.f);
        if (UK != U_NONE) {
            ux = make_float2(__fmul_rn(axo[2 * h], s_now[0]), __fmul_rn(axo[2 * h + 1], s_now[0]));
            uy = make_float2(__fmul_rn(ayo[2 * h], s_now[1]), __fmul_rn(ayo[2 * h + 1], s_now[1]));
        }
        if constexpr (NEQ) phi[h] = collide_pair(v, ux, uy, c);
        else phi[h] = collide_pair_f32(v, ux, uy, c);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[h][i] = v[i];
    }
    if (!live) return;
    if constexpr (NEQ) {
        using P2 = Pair<STORE>;
        using Q = QuadH<STORE>;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            uint2 w;
            w.x = Q::as_u(P2::from_f_raw(out[0][i]));
            w.y = Q::as_u(P2::from_f_raw(out[1][i]));
            *reinterpret_cast<uint2*>(static_cast<unsigned short*>(a.dst) + i * N + cell) = w;
        }
        const float2 p0 = mul2(phi[0], sp2(1.f / SC)), p1 = mul2(phi[1], sp2(1.f / SC));
        *reinterpret_cast<float4*>(a.phi_dst + cell) = make_float4(p0.x, p0.y, p1.x, p1.y);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            *reinterpret_cast<float4*>(static_cast<float*>(a.dst) + i * N + cell) =
                make_float4(out[0][i].x, out[0][i].y, out[1][i].x, out[1][i].y);
    }
}

}  // namespace lbm
