// D3Q15 collision in moment space (Eq. A.2, A.3, A.5) for one node (float)
// or for two nodes at once (float2, paired FP32 instructions of sm_100 and
// later). Included by lbm_device.cuh after the lattice definitions.
//
// The integer maps m = M v and v = M^T a of Eq. A.2 run as butterflies: the
// six axis populations as three sum/difference pairs, the eight corner
// populations (+-1, +-1, +-1) as a three-stage Walsh-Hadamard transform whose
// outputs are exactly the corner parts of the rows 0-8 and of the stress rows
// xy, yz, xz, xyz. About 50 additions per map instead of the ~130 of the
// row-by-row chains.
#pragma once

namespace lbm {

// One arithmetic vocabulary for one node (float) and two nodes (float2). k is
// a constant shared by both nodes; vfmav multiplies two node values.
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vmul(float k, float x) { return __fmul_rn(k, x); }
__device__ __forceinline__ float vfma(float k, float x, float y) { return fmaf(k, x, y); }
__device__ __forceinline__ float vfmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float k, float2 x) { return __fmul2_rn(make_float2(k, k), x); }
__device__ __forceinline__ float2 vfma(float k, float2 x, float2 y) { return __ffma2_rn(make_float2(k, k), x, y); }
__device__ __forceinline__ float2 vfmav(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// m = M v (Eq. A.2). Population order: 0 rest, 1/2 = +-x, 3/4 = +-y, 5/6 = +-z,
// then the corners with e_x alternating +, -, e_y = + for 7, 8, 11, 12 and
// e_z = + for 7 .. 10.
template <class T>
__device__ __forceinline__ void d3q15_moments(const T (&v)[15], T (&m)[15])
{
    const T sx = vadd(v[1], v[2]), ax = vsub(v[1], v[2]);
    const T sy = vadd(v[3], v[4]), ay = vsub(v[3], v[4]);
    const T sz = vadd(v[5], v[6]), az = vsub(v[5], v[6]);
    // corners: over e_x within each (e_y, e_z), then over e_y, then over e_z
    const T p0 = vadd(v[7], v[8]), q0 = vsub(v[7], v[8]);      // (e_y, e_z) = (+, +)
    const T p1 = vadd(v[9], v[10]), q1 = vsub(v[9], v[10]);    // (-, +)
    const T p2 = vadd(v[11], v[12]), q2 = vsub(v[11], v[12]);  // (+, -)
    const T p3 = vadd(v[13], v[14]), q3 = vsub(v[13], v[14]);  // (-, -)
    const T pp0 = vadd(p0, p1), py0 = vsub(p0, p1);
    const T pp1 = vadd(p2, p3), py1 = vsub(p2, p3);
    const T qp0 = vadd(q0, q1), qy0 = vsub(q0, q1);
    const T qp1 = vadd(q2, q3), qy1 = vsub(q2, q3);
    const T h1 = vadd(pp0, pp1), hz = vsub(pp0, pp1);      // sum, sum e_z
    const T hy = vadd(py0, py1), hyz = vsub(py0, py1);     // sum e_y, sum e_y e_z
    const T hx = vadd(qp0, qp1), hxz = vsub(qp0, qp1);     // sum e_x, sum e_x e_z
    const T hxy = vadd(qy0, qy1), hxyz = vsub(qy0, qy1);   // sum e_x e_y, sum e_x e_y e_z
    const T syz = vadd(sy, sz), sa = vadd(sx, syz);
    // row weights at (rest, axis, corner): e^2 - 2 = (-2, -1, 1);
    // (15 e^4 - 55 e^2 + 32) / 2 = (16, -4, 1); (5 e^2 - 13) / 2 = (-, -4, 1)
    m[0] = vadd(vadd(v[0], sa), h1);
    m[1] = vfma(-2.f, v[0], vsub(h1, sa));
    m[2] = vfma(16.f, v[0], vfma(-4.f, sa, h1));
    m[3] = vadd(ax, hx);
    m[4] = vfma(-4.f, ax, hx);
    m[5] = vadd(ay, hy);
    m[6] = vfma(-4.f, ay, hy);
    m[7] = vadd(az, hz);
    m[8] = vfma(-4.f, az, hz);
    m[9] = vfma(2.f, sx, vneg(syz));     // 3 e_x^2 - e^2: (2, -1, -1) on the axes, 0 on corners
    m[10] = vsub(sy, sz);                // e_y^2 - e_z^2
    m[11] = hxy;
    m[12] = hyz;
    m[13] = hxz;
    m[14] = hxyz;
}

// v = M^T a for i >= 1 (and i = 0 when FULL); a_0 is taken as zero when ZERO0.
// Returns v_1 + ... + v_14 in the closed form 6 base + 8 B (exact in exact
// arithmetic), used to close the mass balance through the rest population.
template <class T, bool ZERO0, bool FULL>
__device__ __forceinline__ T d3q15_populations(const T (&a)[15], T (&v)[15])
{
    // axis: base +- X + 2 a9 (x), base +- Y - a9 + a10 (y), base +- Z - a9 - a10 (z)
    const T b12 = vfma(4.f, a[2], a[1]);
    const T base = ZERO0 ? vneg(b12) : vsub(a[0], b12);
    const T X = vfma(-4.f, a[4], a[3]), Y = vfma(-4.f, a[6], a[5]), Z = vfma(-4.f, a[8], a[7]);
    const T Ax = vfma(2.f, a[9], base);
    const T b9 = vsub(base, a[9]);
    const T Ay = vadd(b9, a[10]), Az = vsub(b9, a[10]);
    v[1] = vadd(Ax, X);
    v[2] = vsub(Ax, X);
    v[3] = vadd(Ay, Y);
    v[4] = vsub(Ay, Y);
    v[5] = vadd(Az, Z);
    v[6] = vsub(Az, Z);
    // corners: B + e_x Xd + e_y Yd + e_z Zd + e_x e_y a11 + e_y e_z a12 + e_x e_z a13 + e_x e_y e_z a14
    const T B = ZERO0 ? vadd(a[1], a[2]) : vadd(vadd(a[0], a[1]), a[2]);
    const T Xd = vadd(a[3], a[4]), Yd = vadd(a[5], a[6]), Zd = vadd(a[7], a[8]);
    // coefficients of 1, e_x, e_y, e_x e_y at e_z = +1 (p) and -1 (m)
    const T Pp = vadd(B, Zd), Pm = vsub(B, Zd);
    const T Xp = vadd(Xd, a[13]), Xm = vsub(Xd, a[13]);
    const T Yp = vadd(Yd, a[12]), Ym = vsub(Yd, a[12]);
    const T Wp = vadd(a[11], a[14]), Wm = vsub(a[11], a[14]);
    {
        const T Rp = vadd(Pp, Yp), Rm = vsub(Pp, Yp);   // e_y = +1 / -1
        const T Tp = vadd(Xp, Wp), Tm = vsub(Xp, Wp);   // e_x coefficient at e_y = +1 / -1
        v[7] = vadd(Rp, Tp);
        v[8] = vsub(Rp, Tp);
        v[9] = vadd(Rm, Tm);
        v[10] = vsub(Rm, Tm);
    }
    {
        const T Rp = vadd(Pm, Ym), Rm = vsub(Pm, Ym);
        const T Tp = vadd(Xm, Wm), Tm = vsub(Xm, Wm);
        v[11] = vadd(Rp, Tp);
        v[12] = vsub(Rp, Tp);
        v[13] = vadd(Rm, Tm);
        v[14] = vsub(Rm, Tm);
    }
    if (FULL) v[0] = ZERO0 ? vfma(16.f, a[2], vmul(-2.f, a[1])) : vfma(16.f, a[2], vfma(-2.f, a[1], a[0]));
    return vfma(6.f, base, vmul(8.f, B));
}

// Collision of Eq. A.5 (MRT-A, the only D3Q15 model) for one node or a node
// pair. OFFSET = false: f becomes the post-collision populations f'; OFFSET =
// true: the offsets g = f' - phi (w_i + k_i e_i.u) of the 16-bit forms, from
// moment space as M^-1 (m' - m^eq). Returns phi = m_0.
template <class T, bool OFFSET, class CC>
__device__ __forceinline__ T collide_d3q15(T (&f)[15], T ux, T uy, T uz, const CC& c)
{
    T m[15];
    d3q15_moments(f, m);
    const T phi = m[0];
    const T u[3] = {ux, uy, uz};
    // dl = m - m^eq (Eq. A.3 with c1 = 1 and c2 = -4 of Eq. A.4: linear in u)
    T dl[15];
    dl[1] = vfma(-c.meq1, phi, m[1]);
    dl[2] = vfma(-c.meq2, phi, m[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        dl[3 + 2 * q] = vfmav(vneg(phi), u[q], m[3 + 2 * q]);
        dl[4 + 2 * q] = vfmav(phi, u[q], m[4 + 2 * q]);
    }
#pragma unroll
    for (int k = 9; k < 15; ++k) dl[k] = m[k];
    // m' = m - S dl with the flux rows 3, 5, 7 coupled to rows 4, 6, 8 (Eq. A.5),
    // scaled by 1 / |M_k|^2; the offset form keeps m' - m^eq = dl - S dl, with
    // the relaxation and the scaling folded into c.ro and c.fr
    T a[15];
    if constexpr (OFFSET) {
        a[1] = vmul(c.ro[1], dl[1]);
        a[2] = vmul(c.ro[2], dl[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            T r = vmul(c.fr[6 * q], dl[3]);
            r = vfma(c.fr[6 * q + 1], dl[4], r);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                r = vfma(c.fr[6 * q + 2 * b], dl[3 + 2 * b], r);
                r = vfma(c.fr[6 * q + 2 * b + 1], dl[4 + 2 * b], r);
            }
            a[3 + 2 * q] = r;
            a[4 + 2 * q] = vmul(c.ro[4 + 2 * q], dl[4 + 2 * q]);
        }
#pragma unroll
        for (int k = 9; k < 15; ++k) a[k] = vmul(c.ro[k], dl[k]);
        const T moving = d3q15_populations<T, true, false>(a, f);
        f[0] = vfma(-c.eps0, phi, vneg(moving));   // rest population from the mass balance
        return phi;
    }
    const T(&base)[15] = m;
    a[0] = vmul(1.0f / (float)row_norm2<D3Q15>(0), phi);   // not read by the offset form
    a[1] = vmul(1.0f / (float)row_norm2<D3Q15>(1), vfma(-c.s[1], dl[1], base[1]));
    a[2] = vmul(1.0f / (float)row_norm2<D3Q15>(2), vfma(-c.s[2], dl[2], base[2]));
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        T r = vmul(c.A[3 * q], dl[3]);
        r = vfma(c.C[3 * q], dl[4], r);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            r = vfma(c.A[3 * q + b], dl[3 + 2 * b], r);
            r = vfma(c.C[3 * q + b], dl[4 + 2 * b], r);
        }
        a[3 + 2 * q] = vmul(1.0f / (float)row_norm2<D3Q15>(3 + 2 * q), vsub(base[3 + 2 * q], r));
        a[4 + 2 * q] = vmul(1.0f / (float)row_norm2<D3Q15>(4 + 2 * q),
                            vfma(-c.s[4 + 2 * q], dl[4 + 2 * q], base[4 + 2 * q]));
    }
#pragma unroll
    for (int k = 9; k < 15; ++k)
        a[k] = vmul(1.0f / (float)row_norm2<D3Q15>(k), vfma(-c.s[k], dl[k], base[k]));
    const T moving = d3q15_populations<T, false, false>(a, f);
    f[0] = vsub(phi, moving);   // rest population from the mass balance (see collide in lbm_device.cuh)
    return phi;
}

}  // namespace lbm
