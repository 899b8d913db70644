// Fused stream + collide kernels of the modified-MRT lattice Boltzmann model
// for the convection-diffusion equation (Huang & Wu, arXiv:1404.2363), written
// for sm_103a.
//
// One kernel launch = one time step for every cell:
//   pull-stream f_i(x) = f'_i(x - e_i)                     (Eq. 5, pull form)
//   wall rules on the y = 0 / y = ny-1 nodes                (Sec. 3.2 and variants)
//   m = M f                                                 (Eq. 11-12 / A.2)
//   m' = m - S (m - m^eq(phi, u))  with the modified S      (Eq. 13, 30-31 / A.5)
//   f' = M^-1 m' = M^T diag(1/|M_k|^2) m'                   (Eq. 14, rows orthogonal)
//
// The path is bound by HBM bandwidth (about 1.5 flop per byte), so the design
// goal is the minimum number of DRAM bytes per lattice update with coalesced
// accesses: SoA planes, each warp reads 32 consecutive cells of a plane, the
// x-shifted neighbour reads hit the sectors the neighbouring warps load, and
// the y/z-shifted rows are reused from L2. M, M^-1 and S are compile-time
// integer tables (folded into add/sub chains) and per-solver constants in
// the kernel parameter bank; no tensor cores (a 9x9 or 15x15 integer
// transform per cell is not a dense contraction).
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices. Velocities e_i of Eq. 2 (D2Q9) and Eq. A.1 in the order of the
// moment rows of Eq. A.2 (D3Q15). Moment rows are written as the polynomials
// of e that define them (density, energy, energy squared, momentum, energy
// flux, stress components).
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int DIM = 2;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int M(int k, int i) {
        const int x = ex(i), y = ey(i), e2 = x * x + y * y;
        switch (k) {
            case 0: return 1;
            case 1: return -4 + 3 * e2;
            case 2: return (8 - 21 * e2 + 9 * e2 * e2) / 2;
            case 3: return x;
            case 4: return (-5 + 3 * e2) * x;
            case 5: return y;
            case 6: return (-5 + 3 * e2) * y;
            case 7: return x * x - y * y;
            default: return x * y;
        }
    }
};

struct D3Q15 {
    static constexpr int Q = 15;
    static constexpr int DIM = 3;
    // order: 0, +x, -x, +y, -y, +z, -z, then (+-1,+-1,+-1) with x fastest
    // alternating and z = +1 for i = 7..10, -1 for i = 11..14
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1) ? 1 : (i == 2) ? -1 : (i >= 7) ? ((i % 2) ? 1 : -1) : 0;
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 3) ? 1 : (i == 4) ? -1 : (i >= 7) ? ((((i - 7) / 2) % 2) ? -1 : 1) : 0;
    }
    __host__ __device__ static constexpr int ez(int i) {
        return (i == 5) ? 1 : (i == 6) ? -1 : (i >= 7) ? ((i <= 10) ? 1 : -1) : 0;
    }
    __host__ __device__ static constexpr int M(int k, int i) {
        const int x = ex(i), y = ey(i), z = ez(i), e2 = x * x + y * y + z * z;
        switch (k) {
            case 0: return 1;
            case 1: return e2 - 2;
            case 2: return (15 * e2 * e2 - 55 * e2 + 32) / 2;
            case 3: return x;
            case 4: return (5 * e2 - 13) * x / 2;
            case 5: return y;
            case 6: return (5 * e2 - 13) * y / 2;
            case 7: return z;
            case 8: return (5 * e2 - 13) * z / 2;
            case 9: return 3 * x * x - e2;
            case 10: return y * y - z * z;
            case 11: return x * y;
            case 12: return y * z;
            case 13: return x * z;
            default: return x * y * z;
        }
    }
};

template <class L>
__host__ __device__ constexpr int row_norm2(int k) {
    int s = 0;
    for (int i = 0; i < L::Q; ++i) s += L::M(k, i) * L::M(k, i);
    return s;
}

}  // namespace lbm
#include "lbm_d3q15.cuh"   // D3Q15 moment maps and collision (one node or a node pair)
namespace lbm {

template <class L>
__host__ __device__ constexpr int mirror_y(int i) {
    for (int j = 0; j < L::Q; ++j)
        if (L::ex(j) == L::ex(i) && L::ey(j) == -L::ey(i) && L::ez(j) == L::ez(i)) return j;
    return -1;
}

template <class L>
__host__ __device__ constexpr int opposite(int i) {
    for (int j = 0; j < L::Q; ++j)
        if (L::ex(j) == -L::ex(i) && L::ey(j) == -L::ey(i) && L::ez(j) == -L::ez(i)) return j;
    return -1;
}

// weight class: 0 rest, 1 axis, 2 diagonal
template <class L>
__host__ __device__ constexpr int wclass(int i) {
    const int n = L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i);
    return n == 0 ? 0 : (n == 1 ? 1 : 2);
}

// Arithmetic note: where a product feeds a sum, the kernels use explicitly
// rounded operations (__fmul_rn, fmaf), never left to FMA contraction, so that
// every kernel variant (one node, node pairs, batch) rounds identically.

// e_i . u with e_i in {-1, 0, 1}^3: the non-zero terms added in x, y, z order
template <class L>
__device__ __forceinline__ float e_dot(int i, float ux, float uy, float uz)
{
    const float t[3] = {L::ex(i) > 0 ? ux : -ux, L::ey(i) > 0 ? uy : -uy, L::ez(i) > 0 ? uz : -uz};
    const bool nz[3] = {L::ex(i) != 0, L::ey(i) != 0, L::ez(i) != 0};
    float eu = 0.f;
    bool has = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!nz[a]) continue;
        eu = has ? __fadd_rn(eu, t[a]) : t[a];
        has = true;
    }
    return eu;
}

// f^eq_i / phi = w_i + k_i e_i.u  (equilibria linear in u, Eq. 17)
template <class L>
__device__ __forceinline__ float feq_unit(const Coef& c, int i, float ux, float uy, float uz) {
    const int w = wclass<L>(i);
    if (w == 0) return c.w0;
    const float eu = e_dot<L>(i, ux, uy, uz);
    if (w == 1) return fmaf(c.ka, eu, c.wa);
    return fmaf(c.kd, eu, c.wd);
}

// Full equilibrium f^eq = M^T diag(1/|M_k|^2) m^eq(phi, u), including the u^2
// terms of the MRT-B1/B2 equilibria (used for initial states).
template <class L>
__device__ __forceinline__ void feq_full(const Coef& c, float phi, float ux, float uy, float uz,
                                         float (&fe)[L::Q])
{
    constexpr int Q = L::Q;
    const float u[3] = {ux, uy, uz};
    const float u2 = ux * ux + uy * uy + uz * uz;
    float me[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) me[k] = 0.f;
    me[0] = phi;
    me[1] = fmaf(c.b1, u2, c.meq1) * phi;
    me[2] = fmaf(c.b2, u2, c.meq2) * phi;
#pragma unroll
    for (int a = 0; a < L::DIM; ++a) {
        me[3 + 2 * a] = u[a] * phi;
        me[4 + 2 * a] = -u[a] * phi;
    }
    if (L::Q == 9) {
        me[7] = c.g7 * (ux * ux - uy * uy) * phi;
        me[8] = c.g8 * (ux * uy) * phi;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) me[k] *= 1.0f / (float)row_norm2<L>(k);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) acc = fmaf((float)L::M(k, i), me[k], acc);
        fe[i] = acc;
    }
}

// sum_i w_i v_i for compile-time integer weights w_i = W(i): add/sub chains that
// start from the first non-zero term (0 + x is not folded because of signed zeros).
template <int Q, typename Wf>
__device__ __forceinline__ float int_dot(Wf W, const float* v)
{
    float acc = 0.f;
    bool has = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int w = W(i);
        if (w == 0) continue;
        const float t = (w == 1) ? v[i] : ((w == -1) ? -v[i] : (float)w * v[i]);
        if (!has) {
            acc = t;
            has = true;
        } else if (w == 1) {
            acc += v[i];
        } else if (w == -1) {
            acc -= v[i];
        } else {
            acc = fmaf((float)w, v[i], acc);
        }
    }
    return acc;
}

// ---------------------------------------------------------------------------
// The integer maps m = M v and v = M^T a. For D2Q9 both are evaluated as
// sums and differences of the populations that share |e| (24 operations each
// instead of the 50-58 of the row-by-row chains); D3Q15 as the butterflies of
// lbm_d3q15.cuh.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ void moments(const float (&v)[L::Q], float (&m)[L::Q])
{
    if constexpr (L::Q == 9) {
        // axis pairs (1,3), (2,4) and diagonal pairs (5,7), (6,8) of Eq. 2
        const float sx = v[1] + v[3], ax = v[1] - v[3];
        const float sy = v[2] + v[4], ay = v[2] - v[4];
        const float p57 = v[5] + v[7], d57 = v[5] - v[7];
        const float p68 = v[6] + v[8], d68 = v[6] - v[8];
        const float sa = sx + sy, sd = p57 + p68;      // |e| = 1 and |e|^2 = 2 sums
        const float jx = d57 - d68, jy = d57 + d68;    // diagonal e_x and e_y sums
        m[0] = v[0] + sa + sd;
        m[1] = fmaf(2.f, sd, fmaf(-4.f, v[0], -sa));   // -4, -1, 2
        m[2] = fmaf(-2.f, sa, fmaf(4.f, v[0], sd));    //  4, -2, 1
        m[3] = ax + jx;
        m[4] = fmaf(-2.f, ax, jx);
        m[5] = ay + jy;
        m[6] = fmaf(-2.f, ay, jy);
        m[7] = sx - sy;
        m[8] = p57 - p68;
    } else {
        d3q15_moments<float>(v, m);
    }
}

// v_i = (M^T a)_i for i >= 1 (and i = 0 when FULL); a_0 is taken as zero when
// ZERO0. Returns the sum of v_1 .. v_{Q-1} in a form that is exact in exact
// arithmetic (D2Q9: 4 (A + B), see below), for the mass-balance closure.
template <class L, bool ZERO0, bool FULL>
__device__ __forceinline__ float populations(const float (&a)[L::Q], float (&v)[L::Q])
{
    if constexpr (L::Q == 9) {
        // axis: v = A +- X + P (x) or A +- Y - P (y); diagonal: B +- Xd +- Yd +- R
        const float A = ZERO0 ? fmaf(-2.f, a[2], -a[1]) : fmaf(-2.f, a[2], a[0] - a[1]);
        const float B = ZERO0 ? fmaf(2.f, a[1], a[2]) : fmaf(2.f, a[1], a[0] + a[2]);
        const float X = fmaf(-2.f, a[4], a[3]), Y = fmaf(-2.f, a[6], a[5]);
        const float Xd = a[3] + a[4], Yd = a[5] + a[6];
        const float AP = A + a[7], AM = A - a[7];
        const float BP = B + a[8], BM = B - a[8];
        const float XY = Xd + Yd, XmY = Xd - Yd;
        v[1] = AP + X;
        v[3] = AP - X;
        v[2] = AM + Y;
        v[4] = AM - Y;
        v[5] = BP + XY;
        v[7] = BP - XY;
        v[6] = BM - XmY;
        v[8] = BM + XmY;
        if (FULL) v[0] = ZERO0 ? __fmul_rn(4.f, a[2] - a[1]) : fmaf(4.f, a[2], fmaf(-4.f, a[1], a[0]));
        return __fmul_rn(4.f, A + B);
    } else {
        return d3q15_populations<float, ZERO0, FULL>(a, v);
    }
}

// ---------------------------------------------------------------------------
// Collision in moment space for one node (Eq. 11, 13 with Eq. 31 / A.5, 14).
// On return f holds the post-collision populations f' (OFFSET = false) or
// their offsets from the linear equilibrium, g_i = f'_i - phi (w_i + k_i e_i.u)
// (OFFSET = true, the 16-bit storage forms), computed in moment space as
// g = M^-1 (m' - m^eq_lin). Returns phi = m_0.
// ---------------------------------------------------------------------------
template <class L, bool OFFSET = false, class CC = Coef>
__device__ __forceinline__ float collide(float (&f)[L::Q], float ux, float uy, float uz,
                                         const CC& c)
{
    constexpr int Q = L::Q;
    if constexpr (L::Q == 15) return collide_d3q15<float, OFFSET>(f, ux, uy, uz, c);   // MRT-A only
    float m[Q];
    moments<L>(f, m);
    const float phi = m[0];
    if constexpr (OFFSET && L::Q == 9) {
        // offsets of the 16-bit forms (linear equilibria only): with dl = m - m^eq,
        // a = diag(1/|M_k|^2) (I - S) dl, the rates and scales folded in c.ro, c.fr
        const float dl1 = fmaf(-c.meq1, phi, m[1]), dl2 = fmaf(-c.meq2, phi, m[2]);
        const float dl3 = fmaf(-phi, ux, m[3]), dl4 = fmaf(phi, ux, m[4]);
        const float dl5 = fmaf(-phi, uy, m[5]), dl6 = fmaf(phi, uy, m[6]);
        float a[9];
        a[0] = 0.f;
        a[1] = __fmul_rn(dl1, c.ro[1]);
        a[2] = __fmul_rn(dl2, c.ro[2]);
        a[4] = __fmul_rn(dl4, c.ro[4]);
        a[6] = __fmul_rn(dl6, c.ro[6]);
        a[7] = __fmul_rn(m[7], c.ro[7]);
        a[8] = __fmul_rn(m[8], c.ro[8]);
        a[3] = fmaf(c.fr[0], dl3, fmaf(c.fr[1], dl4, fmaf(c.fr[2], dl5, __fmul_rn(c.fr[3], dl6))));
        a[5] = fmaf(c.fr[4], dl3, fmaf(c.fr[5], dl4, fmaf(c.fr[6], dl5, __fmul_rn(c.fr[7], dl6))));
        f[0] = fmaf(-c.eps0, phi, -populations<L, true, false>(a, f));
        return phi;
    }
    const float u[3] = {ux, uy, uz};
    // dl = m - m^eq_lin (Eq. 15 / A.3 with c1 = 1, c2 from Eq. 16 / A.4: linear in u);
    // d = dl - (u^2 terms of the MRT-B1/B2 equilibria, zero otherwise)
    float dl[Q], d[Q];
    dl[0] = d[0] = 0.f;
    dl[1] = fmaf(-c.meq1, phi, m[1]);
    dl[2] = fmaf(-c.meq2, phi, m[2]);
    d[1] = dl[1];
    d[2] = dl[2];
#pragma unroll
    for (int a = 0; a < L::DIM; ++a) {
        d[3 + 2 * a] = dl[3 + 2 * a] = fmaf(-phi, u[a], m[3 + 2 * a]);
        d[4 + 2 * a] = dl[4 + 2 * a] = fmaf(phi, u[a], m[4 + 2 * a]);
    }
#pragma unroll
    for (int k = 3 + 2 * L::DIM; k < Q; ++k) d[k] = dl[k] = m[k];
    if (c.b1 != 0.f || c.b2 != 0.f || c.g7 != 0.f || c.g8 != 0.f) {   // MRT-B1/B2 only
        float u2 = fmaf(ux, ux, __fmul_rn(uy, uy));
        if (L::DIM == 3) u2 = fmaf(uz, uz, u2);
        d[1] = fmaf(__fmul_rn(-c.b1, u2), phi, dl[1]);
        d[2] = fmaf(__fmul_rn(-c.b2, u2), phi, dl[2]);
        if (L::Q == 9) {
            d[7] = fmaf(__fmul_rn(-c.g7, fmaf(ux, ux, -__fmul_rn(uy, uy))), phi, dl[7]);
            d[8] = fmaf(__fmul_rn(-c.g8, __fmul_rn(ux, uy)), phi, dl[8]);
        }
    }
    // relaxation m' = m - S d; the offset form keeps m' - m^eq_lin = dl - S d
    const float (&base)[Q] = OFFSET ? dl : m;
    float mp[Q];
    mp[0] = OFFSET ? 0.f : phi;
    mp[1] = fmaf(-c.s[1], d[1], base[1]);
    mp[2] = fmaf(-c.s[2], d[2], base[2]);
#pragma unroll
    for (int a = 0; a < L::DIM; ++a) {
        float r = 0.f;
#pragma unroll
        for (int b = 0; b < L::DIM; ++b) {
            r = fmaf(c.A[a * L::DIM + b], d[3 + 2 * b], r);
            r = fmaf(c.C[a * L::DIM + b], d[4 + 2 * b], r);
        }
        mp[3 + 2 * a] = base[3 + 2 * a] - r;
        mp[4 + 2 * a] = fmaf(-c.s[4 + 2 * a], d[4 + 2 * a], base[4 + 2 * a]);
    }
#pragma unroll
    for (int k = 3 + 2 * L::DIM; k < Q; ++k) mp[k] = fmaf(-c.s[k], d[k], base[k]);
    // f' = M^T diag(1 / |row|^2) m'
#pragma unroll
    for (int k = 0; k < Q; ++k) mp[k] = __fmul_rn(mp[k], 1.0f / (float)row_norm2<L>(k));
    const float moving = populations<L, OFFSET, false>(mp, f);
    // The rest population closes the mass balance: sum_i f'_i = m'_0 = phi
    // (row 0 of M^-1 m'). Taking it from the moving populations keeps FP32
    // rounding of the 1/|M_0|^2 factor from biasing the total mass. For the
    // offsets, sum_i g_i = -phi eps0 balances the FP32 weights of the decode,
    // which sum to 1 + eps0 (else the mass would drift by phi eps0 per step).
    if constexpr (OFFSET) f[0] = fmaf(-c.eps0, phi, -moving);   // see Coef::eps0
    else f[0] = phi - moving;
    return phi;
}

// ---------------------------------------------------------------------------
// Storage helpers
// ---------------------------------------------------------------------------
template <int S> struct StT;
template <> struct StT<ST_F32> { using T = float; };
template <> struct StT<ST_F16> { using T = __half; };
template <> struct StT<ST_BF16> { using T = __nv_bfloat16; };

// FP16 offsets are stored multiplied by 2^11 (exact): the non-equilibrium
// offsets of dilute regions (phi ~ 1e-4) then stay in FP16's normal range
// instead of its subnormals, while |g| up to 32 remains representable.
constexpr float F16_SCALE = 2048.0f;

__device__ __forceinline__ float ldg_f(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_f(const __half* p) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p)))) *
           (1.0f / F16_SCALE);
}
__device__ __forceinline__ float ldg_f(const __nv_bfloat16* p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ void st_f(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_f(__half* p, float v) { *p = __float2half_rn(v * F16_SCALE); }
__device__ __forceinline__ void st_f(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Schedule multipliers s(k) (t mod sched_len), 1 when there is no schedule.
__device__ __forceinline__ void sched_at(const float* sched, long long len, long long k, int dim, float* s)
{
    s[0] = s[1] = s[2] = 1.f;
    if (sched != nullptr && len > 0) {
        long long r = k % len;
        if (r < 0) r += len;
        for (int d = 0; d < dim; ++d) s[d] = __ldg(sched + r * dim + d);
    }
}

__device__ __forceinline__ void sched_at(const StepArgs& a, long long k, int dim, float* s)
{
    sched_at(a.sched, a.sched_len, k, dim, s);
}

// the same from a row computed on the host (row < 0: no schedule)
__device__ __forceinline__ void sched_row_at(const float* sched, int row, int dim, float* s)
{
    s[0] = s[1] = s[2] = 1.f;
    if (row >= 0)
        for (int d = 0; d < dim; ++d) s[d] = __ldg(sched + row * dim + d);
}

// u(x, k) = a(x) s(k) for a field, a(y) s(k) for a row profile, 0 otherwise.
template <int UK, int DIM>
__device__ __forceinline__ void vel_at_p(const float* ua, long long ncell, int ny, long long cell, int y,
                                         const float* s, float& ux, float& uy, float& uz)
{
    ux = uy = uz = 0.f;
    if (UK == U_FIELD) {
        ux = __fmul_rn(__ldg(ua + cell), s[0]);
        uy = __fmul_rn(__ldg(ua + ncell + cell), s[1]);
        if (DIM == 3) uz = __fmul_rn(__ldg(ua + 2 * ncell + cell), s[2]);
    } else if (UK == U_ROW) {
        ux = __fmul_rn(__ldg(ua + y), s[0]);
        uy = __fmul_rn(__ldg(ua + ny + y), s[1]);
        if (DIM == 3) uz = __fmul_rn(__ldg(ua + 2 * ny + y), s[2]);
    }
}

template <int UK, int DIM>
__device__ __forceinline__ void vel_at(const StepArgs& a, long long cell, int y, const float* s,
                                       float& ux, float& uy, float& uz)
{
    vel_at_p<UK, DIM>(a.ua, a.ncell, a.ny, cell, y, s, ux, uy, uz);
}

// ---------------------------------------------------------------------------
// The fused step kernel.
// grid = (ceil(nx / (blockDim.x * VEC)), ny, nz); thread handles the cells
// x = (blockIdx.x * VEC + j) * blockDim.x + threadIdx.x, j < VEC.
// ---------------------------------------------------------------------------
// IX is the index type: int when every plane offset fits in 31 bits (fewer
// address instructions), long long otherwise.
template <int UK, int DIM, typename IX>
__device__ __forceinline__ void vel_ix(const StepArgs& a, IX N, IX cell, int y, const float* s,
                                       float& ux, float& uy, float& uz)
{
    ux = uy = uz = 0.f;
    if (UK == U_FIELD) {
        ux = __fmul_rn(__ldg(a.ua + cell), s[0]);
        uy = __fmul_rn(__ldg(a.ua + N + cell), s[1]);
        if (DIM == 3) uz = __fmul_rn(__ldg(a.ua + 2 * N + cell), s[2]);
    } else if (UK == U_ROW) {
        ux = __fmul_rn(__ldg(a.ua + y), s[0]);
        uy = __fmul_rn(__ldg(a.ua + a.ny + y), s[1]);
        if (DIM == 3) uz = __fmul_rn(__ldg(a.ua + 2 * a.ny + y), s[2]);
    }
}

template <class L, int STORE, int UK, bool WALLS, int VEC, typename IX>
__global__ void __launch_bounds__(256) k_step(const StepArgs a)
{
    using T = typename StT<STORE>::T;
    constexpr int Q = L::Q;
    constexpr bool NEQ = (STORE != ST_F32);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int y = blockIdx.y, z = blockIdx.z;
    const IX N = (IX)a.ncell;
    const T* __restrict__ src = static_cast<const T*>(a.src);
    T* __restrict__ dst = static_cast<T*>(a.dst);

    // source rows for e_y = -1, 0, +1 (index ey + 1): row y - e_y, periodic
    const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
    const int zs[3] = {z + 1 == nz ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};

    float s_now[3], s_prev[3];
    if (UK != U_NONE) {
        sched_row_at(a.sched, a.srow_now, L::DIM, s_now);
        sched_row_at(a.sched, a.srow_prev, L::DIM, s_prev);
    }

    float f[VEC][Q];
    IX cell[VEC];
    bool live[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const int x = (blockIdx.x * VEC + j) * blockDim.x + threadIdx.x;
        live[j] = x < nx;
        const int xc = live[j] ? x : nx - 1;
        const int xs[3] = {xc + 1 == nx ? 0 : xc + 1, xc, xc == 0 ? nx - 1 : xc - 1};
        cell[j] = (IX)xc + (IX)nx * ((IX)y + (IX)ny * (IX)z);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const IX sc = (IX)xs[L::ex(i) + 1] + (IX)nx * ((IX)ys[L::ey(i) + 1] + (IX)ny * (IX)zs[L::ez(i) + 1]);
            float v = ldg_f(src + (IX)i * N + sc);
            if (NEQ) {
                float ux, uy, uz;
                vel_ix<UK, L::DIM, IX>(a, N, sc, ys[L::ey(i) + 1], s_prev, ux, uy, uz);
                v = fmaf(__ldg(a.phi_src + sc), feq_unit<L>(a.c, i, ux, uy, uz), v);
            }
            f[j][i] = v;
        }
    }

#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        if (WALLS) {
            const bool lo = (y == 0) && a.bc_lo != BC_PERIODIC;
            const bool hi = (y == ny - 1) && a.bc_hi != BC_PERIODIC;
            if (lo || hi) {
                const int kind = lo ? a.bc_lo : a.bc_hi;
                const int inward = lo ? 1 : -1;   // e_y of the populations entering from the wall
                if (kind == BC_NOFLUX) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ey(i) != 0 && ((L::ey(i) == 1) == lo)) f[j][i] = f[j][mirror_y<L>(i)];
                } else if (kind == BC_BOUNCE) {
                    float ux = 0.f, uy = 0.f, uz = 0.f;
                    if (NEQ) vel_ix<UK, L::DIM, IX>(a, N, cell[j], y, s_prev, ux, uy, uz);
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ey(i) != 0 && ((L::ey(i) == 1) == lo)) {
                            const int o = opposite<L>(i);
                            float v = ldg_f(src + (IX)o * N + cell[j]);
                            if (NEQ) v = fmaf(__ldg(a.phi_src + cell[j]), feq_unit<L>(a.c, o, ux, uy, uz), v);
                            f[j][i] = v;
                        }
                } else {  // Dirichlet
                    float ux, uy, uz;
                    vel_ix<UK, L::DIM, IX>(a, N, cell[j], y, s_prev, ux, uy, uz);
                    float known = 0.f, wk = 0.f;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (L::ey(i) == inward) wk += feq_unit<L>(a.c, i, ux, uy, uz);
                        else known += f[j][i];
                    }
                    const float phiw = lo ? a.phiw_lo : a.phiw_hi;
                    const float ps = (phiw - known) / wk;
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ey(i) == inward) f[j][i] = __fmul_rn(ps, feq_unit<L>(a.c, i, ux, uy, uz));
                }
            }
        }
        float ux, uy, uz;
        vel_ix<UK, L::DIM, IX>(a, N, cell[j], y, s_now, ux, uy, uz);
        const float phi = collide<L, NEQ>(f[j], ux, uy, uz, a.c);
        if (!live[j]) continue;
#pragma unroll
        for (int i = 0; i < Q; ++i) st_f(dst + (IX)i * N + cell[j], f[j][i]);
        if (NEQ) a.phi_dst[cell[j]] = phi;
    }
}

// ---------------------------------------------------------------------------
// The step with walls on the x (and z) faces as well (any storage, one node per
// thread; the other kernels take periodic x and z). For each population i the
// pull source x - e_i is checked against every face; a source beyond a face
// whose axis is not periodic is not read:
//   - if one of the faces it lies beyond is BOUNCEBACK, f_i = f'_opp(i) of the
//     node itself (halfway bounce-back);
//   - then, if it lies beyond NOFLUX_NODE faces, f_i takes the value of the
//     population reflected in the axes of those faces (the Sec. 3.2 mirror rule,
//     applied per axis; at an edge of two Neumann faces, reflected in both);
//   - Dirichlet (y faces only) replaces every population entering from beyond
//     the y wall, as in k_step.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ int reflect_mask(int i, int mask)
{
    const int e[3] = {(mask & 1) ? -L::ex(i) : L::ex(i), (mask & 2) ? -L::ey(i) : L::ey(i),
                      (mask & 4) ? -L::ez(i) : L::ez(i)};
    int r = i;
#pragma unroll
    for (int j = 0; j < L::Q; ++j)
        if (L::ex(j) == e[0] && L::ey(j) == e[1] && L::ez(j) == e[2]) r = j;
    return r;
}

template <class L, int STORE, int UK, typename IX>
__global__ void __launch_bounds__(256) k_step_box(const StepArgs a)
{
    using T = typename StT<STORE>::T;
    constexpr int Q = L::Q;
    constexpr bool NEQ = (STORE != ST_F32);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const IX N = (IX)a.ncell;
    const T* __restrict__ src = static_cast<const T*>(a.src);
    T* __restrict__ dst = static_cast<T*>(a.dst);
    const int pos[3] = {x, y, z}, n[3] = {nx, ny, nz};
    const int klo[3] = {a.bcx_lo, a.bc_lo, a.bcz_lo}, khi[3] = {a.bcx_hi, a.bc_hi, a.bcz_hi};
    const IX cell = (IX)x + (IX)nx * ((IX)y + (IX)ny * (IX)z);
    float s_now[3], s_prev[3];
    if (UK != U_NONE) {
        sched_row_at(a.sched, a.srow_now, L::DIM, s_now);
        sched_row_at(a.sched, a.srow_prev, L::DIM, s_prev);
    }
    float uxp = 0.f, uyp = 0.f, uzp = 0.f;   // u(k - 1) at the node (bounce-back decode, Dirichlet)
    vel_ix<UK, L::DIM, IX>(a, N, cell, y, s_prev, uxp, uyp, uzp);
    float w[Q];
    int nf[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        int sp[3];
        bool out = false, bb = false;
        nf[i] = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sp[d] = pos[d] - e[d];
            if (e[d] == 0) continue;
            if (klo[d] == BC_PERIODIC) {
                sp[d] = sp[d] < 0 ? sp[d] + n[d] : (sp[d] >= n[d] ? sp[d] - n[d] : sp[d]);
            } else if (sp[d] < 0 || sp[d] >= n[d]) {
                const int kind = sp[d] < 0 ? klo[d] : khi[d];
                out = true;
                bb = bb || kind == BC_BOUNCE;
                if (kind == BC_NOFLUX) nf[i] |= 1 << d;
            }
        }
        float v = 0.f;
        if (!out) {
            const IX sc = (IX)sp[0] + (IX)nx * ((IX)sp[1] + (IX)ny * (IX)sp[2]);
            v = ldg_f(src + (IX)i * N + sc);
            if (NEQ) {
                float ux, uy, uz;
                vel_ix<UK, L::DIM, IX>(a, N, sc, sp[1], s_prev, ux, uy, uz);
                v = fmaf(__ldg(a.phi_src + sc), feq_unit<L>(a.c, i, ux, uy, uz), v);
            }
        } else if (bb) {
            const int o = opposite<L>(i);
            v = ldg_f(src + (IX)o * N + cell);
            if (NEQ) v = fmaf(__ldg(a.phi_src + cell), feq_unit<L>(a.c, o, uxp, uyp, uzp), v);
        }
        w[i] = v;
    }
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        f[i] = w[i];
        if (nf[i]) {
            const int j = reflect_mask<L>(i, nf[i]);
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (k == j) f[i] = w[k];
        }
    }
    const bool lo = y == 0 && a.bc_lo == BC_DIRICHLET, hi = y == ny - 1 && a.bc_hi == BC_DIRICHLET;
    if (lo || hi) {
        const int inward = lo ? 1 : -1;
        float known = 0.f, wk = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (L::ey(i) == inward) wk += feq_unit<L>(a.c, i, uxp, uyp, uzp);
            else known += f[i];
        }
        const float ps = ((lo ? a.phiw_lo : a.phiw_hi) - known) / wk;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::ey(i) == inward) f[i] = __fmul_rn(ps, feq_unit<L>(a.c, i, uxp, uyp, uzp));
    }
    float ux, uy, uz;
    vel_ix<UK, L::DIM, IX>(a, N, cell, y, s_now, ux, uy, uz);
    const float phi = collide<L, NEQ>(f, ux, uy, uz, a.c);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_f(dst + (IX)i * N + cell, f[i]);
    if (NEQ) a.phi_dst[cell] = phi;
}

template <class L, int STORE, int UK>
__global__ void k_init(const StepArgs a, const float* __restrict__ phi0)
{
    using T = typename StT<STORE>::T;
    T* dst = static_cast<T*>(a.dst);
    float s0[3];
    sched_at(a, 0, L::DIM, s0);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((c / a.nx) % a.ny);
        float ux, uy, uz;
        vel_at<UK, L::DIM>(a, c, y, s0, ux, uy, uz);
        const float p = phi0[c];
        float fe[L::Q];
        feq_full<L>(a.c, p, ux, uy, uz, fe);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) st_f(dst + (long long)i * a.ncell + c, (STORE == ST_F32) ? fe[i] : 0.f);
        if (STORE != ST_F32) a.phi_dst[c] = p;
    }
}

template <class L, int STORE>
__global__ void k_phi(const StepArgs a, float* __restrict__ out)
{
    using T = typename StT<STORE>::T;
    const T* src = static_cast<const T*>(a.src);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        if (STORE != ST_F32) {
            out[c] = a.phi_src[c];
        } else {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) s += ldg_f(src + (long long)i * a.ncell + c);
            out[c] = s;
        }
    }
}

// Deterministic FP64 sum of phi: pass 1 writes one partial per block (fixed
// grid-stride order, fixed shared-memory tree), pass 2 sums the partials in
// index order in one block.
template <class L, int STORE>
__global__ void __launch_bounds__(256) k_sum1(const StepArgs a, double* __restrict__ partials)
{
    using T = typename StT<STORE>::T;
    const T* src = static_cast<const T*>(a.src);
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        if (STORE != ST_F32) {
            acc += (double)a.phi_src[c];
        } else {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) s += (double)ldg_f(src + (long long)i * a.ncell + c);
            acc += s;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}


}  // namespace lbm
