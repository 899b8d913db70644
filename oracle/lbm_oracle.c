/*
 * FP64 CPU oracle for the modified multiple-relaxation-time lattice Boltzmann
 * model of the convection-diffusion equation (Huang & Wu, arXiv:1404.2363).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. The GPU library neither
 * links, includes nor calls anything here, and this file shares no header,
 * table, constant generator or helper with it.
 *
 * The oracle runs the paper's algorithm literally, in the paper's order:
 *   collision in moment space (Eq. 11, 13, 14) with the dense relaxation
 *   matrix S of Eq. 31 (modified, MRT-A) or Eq. 24 (unmodified, MRT-B1/B2/B3),
 *   then streaming in push form (Eq. 5), then the wall rules.
 * The state held between steps is the pre-collision distribution f(x, t).
 * M is typed from Eq. 12 (D2Q9) / Eq. A.2 (D3Q15); M^-1 is obtained by
 * numerically inverting M (Gauss-Jordan), not from any closed form.
 *
 * Lattice units: dx = dt = c = 1.  Cell index: x + nx*(y + ny*z).
 * Distribution layout: f[i*ncell + cell] (one plane per direction).
 * Velocity layout: u[a*ncell + cell], a = 0..dim-1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 15

enum { ORC_MRT_A = 0, ORC_MRT_B1 = 1, ORC_MRT_B2 = 2, ORC_MRT_B3 = 3 };
enum { ORC_PERIODIC = 0, ORC_NOFLUX_NODE = 1, ORC_BOUNCEBACK = 2, ORC_DIRICHLET = 3 };

/* Parameters of one run.  The two y faces carry bc_lo / bc_hi (any wall kind);
 * the x faces bcx_lo / bcx_hi and the z faces bcz_lo / bcz_hi (D3Q15) are
 * periodic, NOFLUX_NODE or BOUNCEBACK.  s[k] are the diagonal rates of S; the
 * flux rows (3, 5 in D2Q9; 3, 5, 7 in D3Q15) take the block A instead. */
typedef struct {
    int32_t q;          /* 9 or 15 */
    int32_t model;      /* ORC_MRT_* (B models exist for D2Q9 only) */
    int64_t nx, ny, nz; /* nz = 1 for D2Q9 */
    int32_t bc_lo, bc_hi;
    double phi_w_lo, phi_w_hi; /* Dirichlet wall values */
    double alpha1, alpha2;     /* free equilibrium parameters (Eq. 15, A.3) */
    double s[15];              /* diagonal relaxation rates s_0..s_{q-1} */
    double A[9];               /* flux block of S, row-major dim x dim */
    int32_t nthreads;          /* OpenMP threads (<= 0: library default) */
    int32_t bcx_lo, bcx_hi;    /* x faces */
    int32_t bcz_lo, bcz_hi;    /* z faces (D3Q15) */
} orc_params;

typedef struct {
    int q, dim;
    int e[ORC_MAXQ][3];
    double M[ORC_MAXQ][ORC_MAXQ];
    double Minv[ORC_MAXQ][ORC_MAXQ];
    double S[ORC_MAXQ][ORC_MAXQ];
} orc_lattice;

/* ---------------------------------------------------------------------- */
/* Transformation matrices, typed from the paper.                          */
/* ---------------------------------------------------------------------- */

/* Eq. 12: D2Q9 M for c = 1. Rows: rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy */
static const int M_D2Q9[9][9] = {
    { 1,  1,  1,  1,  1, 1,  1,  1,  1},
    {-4, -1, -1, -1, -1, 2,  2,  2,  2},
    { 4, -2, -2, -2, -2, 1,  1,  1,  1},
    { 0,  1,  0, -1,  0, 1, -1, -1,  1},
    { 0, -2,  0,  2,  0, 1, -1, -1,  1},
    { 0,  0,  1,  0, -1, 1,  1, -1, -1},
    { 0,  0, -2,  0,  2, 1,  1, -1, -1},
    { 0,  1, -1,  1, -1, 0,  0,  0,  0},
    { 0,  0,  0,  0,  0, 1, -1,  1, -1},
};

/* Eq. A.2: D3Q15 M for c = 1. Rows: rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z,
 * 3p_xx, p_ww, p_xy, p_yz, p_xz, m_xyz */
static const int M_D3Q15[15][15] = {
    { 1,  1,  1,  1,  1,  1,  1, 1,  1,  1,  1,  1,  1,  1,  1},
    {-2, -1, -1, -1, -1, -1, -1, 1,  1,  1,  1,  1,  1,  1,  1},
    {16, -4, -4, -4, -4, -4, -4, 1,  1,  1,  1,  1,  1,  1,  1},
    { 0,  1, -1,  0,  0,  0,  0, 1, -1,  1, -1,  1, -1,  1, -1},
    { 0, -4,  4,  0,  0,  0,  0, 1, -1,  1, -1,  1, -1,  1, -1},
    { 0,  0,  0,  1, -1,  0,  0, 1,  1, -1, -1,  1,  1, -1, -1},
    { 0,  0,  0, -4,  4,  0,  0, 1,  1, -1, -1,  1,  1, -1, -1},
    { 0,  0,  0,  0,  0,  1, -1, 1,  1,  1,  1, -1, -1, -1, -1},
    { 0,  0,  0,  0,  0, -4,  4, 1,  1,  1,  1, -1, -1, -1, -1},
    { 0,  2,  2, -1, -1, -1, -1, 0,  0,  0,  0,  0,  0,  0,  0},
    { 0,  0,  0,  1,  1, -1, -1, 0,  0,  0,  0,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  0,  0, 1, -1, -1,  1,  1, -1, -1,  1},
    { 0,  0,  0,  0,  0,  0,  0, 1,  1, -1, -1, -1, -1,  1,  1},
    { 0,  0,  0,  0,  0,  0,  0, 1, -1,  1, -1, -1,  1, -1,  1},
    { 0,  0,  0,  0,  0,  0,  0, 1, -1, -1,  1, -1,  1,  1, -1},
};

/* Gauss-Jordan inversion with partial pivoting (n <= 15). Returns 0 on success. */
static int invert(int n, double a[ORC_MAXQ][ORC_MAXQ], double inv[ORC_MAXQ][ORC_MAXQ])
{
    double w[ORC_MAXQ][2 * ORC_MAXQ];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            w[r][c] = (c < n) ? a[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r][col]) > fabs(w[piv][col])) piv = r;
        if (w[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col][c]; w[col][c] = w[piv][c]; w[piv][c] = t;
            }
        double d = w[col][col];
        for (int c = 0; c < 2 * n; ++c) w[col][c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = w[r][col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r][c] -= fct * w[col][c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r][c] = w[r][c + n];
    return 0;
}

/* The modified relaxation matrix of Eq. 31 (D2Q9) or Eq. A.5 (D3Q15), or the
 * unmodified one of Eq. 24 (D2Q9, the MRT-B models). */
static void build_S(orc_lattice* L, const orc_params* p)
{
    memset(L->S, 0, sizeof(L->S));
    for (int k = 0; k < L->q; ++k) L->S[k][k] = p->s[k];
    if (L->q == 9) {
        const double sxx = p->A[0], sxy = p->A[1], syx = p->A[2], syy = p->A[3];
        const double s4 = p->s[4], s6 = p->s[6];
        L->S[3][3] = sxx; L->S[3][5] = sxy;
        L->S[5][3] = syx; L->S[5][5] = syy;
        if (p->model == ORC_MRT_A) { /* Eq. 30a, 30b */
            L->S[3][4] = (sxx / 2.0 - 1.0) * s4;
            L->S[3][6] = (sxy / 2.0) * s6;
            L->S[5][4] = (syx / 2.0) * s4;
            L->S[5][6] = (syy / 2.0 - 1.0) * s6;
        }
    } else {
        const double sxx = p->A[0], sxy = p->A[1], sxz = p->A[2];
        const double syx = p->A[3], syy = p->A[4], syz = p->A[5];
        const double szx = p->A[6], szy = p->A[7], szz = p->A[8];
        const double s4 = p->s[4], s6 = p->s[6], s8 = p->s[8];
        /* Eq. A.5 row 3 */
        L->S[3][3] = sxx; L->S[3][4] = (sxx / 2.0 - 1.0) * s4;
        L->S[3][5] = sxy; L->S[3][6] = (sxy / 2.0) * s6;
        L->S[3][7] = sxz; L->S[3][8] = (sxz / 2.0) * s8;
        /* row 5 */
        L->S[5][3] = syx; L->S[5][4] = (syx / 2.0) * s4;
        L->S[5][5] = syy; L->S[5][6] = (syy / 2.0 - 1.0) * s6;
        L->S[5][7] = syz; L->S[5][8] = (syz / 2.0) * s8;
        /* row 7 */
        L->S[7][3] = szx; L->S[7][4] = (szx / 2.0) * s4;
        L->S[7][5] = szy; L->S[7][6] = (szy / 2.0) * s6;
        L->S[7][7] = szz; L->S[7][8] = (szz / 2.0 - 1.0) * s8;
    }
}

static int build_lattice(orc_lattice* L, const orc_params* p)
{
    memset(L, 0, sizeof(*L));
    L->q = p->q;
    if (p->q == 9) {
        L->dim = 2;
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 9; ++c) L->M[r][c] = M_D2Q9[r][c];
        /* Eq. 2 with c = 1 */
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < 9; ++i) {
            double ex = 0.0, ey = 0.0;
            if (i >= 1 && i <= 4) {
                ex = cos((i - 1) * pi / 2.0);
                ey = sin((i - 1) * pi / 2.0);
            } else if (i >= 5) {
                ex = sqrt(2.0) * cos((2 * i - 9) * pi / 4.0);
                ey = sqrt(2.0) * sin((2 * i - 9) * pi / 4.0);
            }
            L->e[i][0] = (int)lround(ex);
            L->e[i][1] = (int)lround(ey);
            L->e[i][2] = 0;
        }
    } else if (p->q == 15) {
        L->dim = 3;
        for (int r = 0; r < 15; ++r)
            for (int c = 0; c < 15; ++c) L->M[r][c] = M_D3Q15[r][c];
        /* Eq. A.1 gives the set; the order is the one the rows j_x, j_y, j_z
         * of Eq. A.2 fix (row 3 is e_x, row 5 is e_y, row 7 is e_z). */
        for (int i = 0; i < 15; ++i) {
            L->e[i][0] = M_D3Q15[3][i];
            L->e[i][1] = M_D3Q15[5][i];
            L->e[i][2] = M_D3Q15[7][i];
        }
        if (p->model != ORC_MRT_A) return -2;
    } else {
        return -1;
    }
    /* x and z faces: both periodic or both walls, NOFLUX_NODE or BOUNCEBACK;
     * D2Q9 has no z faces */
    const int32_t fx[2] = {p->bcx_lo, p->bcx_hi}, fz[2] = {p->bcz_lo, p->bcz_hi};
    for (int k = 0; k < 2; ++k) {
        if (fx[k] < ORC_PERIODIC || fx[k] > ORC_BOUNCEBACK) return -5;
        if (fz[k] < ORC_PERIODIC || fz[k] > ORC_BOUNCEBACK) return -5;
    }
    if ((fx[0] == ORC_PERIODIC) != (fx[1] == ORC_PERIODIC)) return -5;
    if ((fz[0] == ORC_PERIODIC) != (fz[1] == ORC_PERIODIC)) return -5;
    if (p->q == 9 && fz[0] != ORC_PERIODIC) return -5;
    if (invert(L->q, L->M, L->Minv) != 0) return -3;
    build_S(L, p);
    return 0;
}

/* Equilibrium moments m^eq(phi, u).
 *   MRT-A (and B3 via its alpha values): Eq. 15 with c1 = 1, c2 = -2 (Eq. 16)
 *   MRT-B1: Eq. 38;  MRT-B2: Eq. 39;  MRT-B3: Eq. 37 with the unmodified S
 *   D3Q15: Eq. A.3 with c1 = 1, c2 = -4 (Eq. A.4). */
static void meq(const orc_lattice* L, const orc_params* p, double phi, const double u[3],
                double m[ORC_MAXQ])
{
    for (int k = 0; k < L->q; ++k) m[k] = 0.0;
    if (L->q == 9) {
        const double ux = u[0], uy = u[1], u2 = ux * ux + uy * uy;
        if (p->model == ORC_MRT_A || p->model == ORC_MRT_B3) {
            const double a1 = (p->model == ORC_MRT_B3) ? -8.0 : p->alpha1;
            const double a2 = (p->model == ORC_MRT_B3) ? 8.0 : p->alpha2;
            const double c1 = 1.0, c2 = -2.0 * c1;
            m[0] = phi;
            m[1] = 0.25 * a1 * phi;
            m[2] = 0.25 * a2 * phi;
            m[3] = c1 * phi * ux;
            m[5] = c1 * phi * uy;
            m[4] = 0.5 * c2 * phi * ux;
            m[6] = 0.5 * c2 * phi * uy;
            m[7] = 0.0;
            m[8] = 0.0;
        } else {
            m[0] = phi;
            m[1] = phi * (-2.0 + 3.0 * u2);
            m[2] = phi * ((p->model == ORC_MRT_B1 ? 1.0 : 2.0) - 3.0 * u2);
            m[3] = phi * ux;
            m[4] = -phi * ux;
            m[5] = phi * uy;
            m[6] = -phi * uy;
            m[7] = phi * (ux * ux - uy * uy);
            m[8] = phi * ux * uy;
        }
    } else {
        const double c1 = 1.0, c2 = -4.0 * c1;
        m[0] = phi;
        m[1] = 5.0 / 6.0 * p->alpha1 * phi;
        m[2] = p->alpha2 / 24.0 * phi;
        m[3] = c1 * phi * u[0];
        m[5] = c1 * phi * u[1];
        m[7] = c1 * phi * u[2];
        m[4] = 0.25 * c2 * phi * u[0];
        m[6] = 0.25 * c2 * phi * u[1];
        m[8] = 0.25 * c2 * phi * u[2];
    }
}

/* d m^eq / d u_a at unit phi (column a of the velocity Jacobian). */
static void dmeq_du(const orc_lattice* L, const orc_params* p, const double u[3], int a,
                    double d[ORC_MAXQ])
{
    for (int k = 0; k < L->q; ++k) d[k] = 0.0;
    if (L->q == 9) {
        const double ux = u[0], uy = u[1];
        const int fr = (a == 0) ? 3 : 5;
        d[fr] = 1.0;
        d[fr + 1] = -1.0;
        if (p->model == ORC_MRT_B1 || p->model == ORC_MRT_B2) {
            const double ua = (a == 0) ? ux : uy;
            d[1] = 6.0 * ua;
            d[2] = -6.0 * ua;
            d[7] = (a == 0) ? 2.0 * ux : -2.0 * uy;
            d[8] = (a == 0) ? uy : ux;
        }
    } else {
        const int fr = 3 + 2 * a;
        d[fr] = 1.0;
        d[fr + 1] = -1.0;
    }
}

static void matvec(int n, const double A[ORC_MAXQ][ORC_MAXQ], const double* x, double* y)
{
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc += A[r][c] * x[c];
        y[r] = acc;
    }
}

static void matTvec(int n, const double A[ORC_MAXQ][ORC_MAXQ], const double* x, double* y)
{
    for (int c = 0; c < n; ++c) {
        double acc = 0.0;
        for (int r = 0; r < n; ++r) acc += A[r][c] * x[r];
        y[c] = acc;
    }
}

/* One collision at a node: Eq. 11, then Eq. 13 (dense S), then Eq. 14. */
static void collide_node(const orc_lattice* L, const orc_params* p, const double* f,
                         const double u[3], double* fout)
{
    const int q = L->q;
    double m[ORC_MAXQ], me[ORC_MAXQ], dm[ORC_MAXQ], sd[ORC_MAXQ], mp[ORC_MAXQ];
    matvec(q, L->M, f, m);                 /* Eq. 11 */
    meq(L, p, m[0], u, me);                /* phi = m_0 (Eq. 8, 15a) */
    for (int k = 0; k < q; ++k) dm[k] = m[k] - me[k];
    matvec(q, L->S, dm, sd);
    for (int k = 0; k < q; ++k) mp[k] = m[k] - sd[k]; /* Eq. 13 */
    matvec(q, L->Minv, mp, fout);          /* Eq. 14 */
}

static inline int64_t wrap(int64_t v, int64_t n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

static int64_t ncells(const orc_params* p) { return p->nx * p->ny * p->nz; }

static void get_u(const orc_lattice* L, const double* u, int64_t nc, int64_t cell, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    if (!u) return;
    for (int a = 0; a < L->dim; ++a) out[a] = u[a * nc + cell];
}

static int mirror_y(const orc_lattice* L, int i)
{
    for (int j = 0; j < L->q; ++j)
        if (L->e[j][0] == L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == L->e[i][2])
            return j;
    return -1;
}

static int opposite(const orc_lattice* L, int i)
{
    for (int j = 0; j < L->q; ++j)
        if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2])
            return j;
    return -1;
}

/* Wall kind of face (axis a, side 0 = low / 1 = high). */
static int face_kind(const orc_params* p, int a, int side)
{
    if (a == 0) return side ? p->bcx_hi : p->bcx_lo;
    if (a == 1) return side ? p->bc_hi : p->bc_lo;
    return side ? p->bcz_hi : p->bcz_lo;
}

/* Whether node (x, y, z) lies on a face that is not periodic. */
static int on_wall(const orc_params* p, int64_t x, int64_t y, int64_t z)
{
    return (p->bcx_lo != ORC_PERIODIC && (x == 0 || x == p->nx - 1)) ||
           (p->bc_lo != ORC_PERIODIC && (y == 0 || y == p->ny - 1)) ||
           (p->bcz_lo != ORC_PERIODIC && (z == 0 || z == p->nz - 1));
}

static int any_wall(const orc_params* p)
{
    return p->bc_lo != ORC_PERIODIC || p->bcx_lo != ORC_PERIODIC || p->bcz_lo != ORC_PERIODIC;
}

/* The population whose velocity is e_i reflected in the axes whose bit is set in mask. */
static int reflect(const orc_lattice* L, int i, int mask)
{
    int e[3];
    for (int a = 0; a < 3; ++a) e[a] = (mask >> a & 1) ? -L->e[i][a] : L->e[i][a];
    for (int j = 0; j < L->q; ++j)
        if (L->e[j][0] == e[0] && L->e[j][1] == e[1] && L->e[j][2] == e[2]) return j;
    return -1;
}

/* For population i at node (x, y, z): the faces its pull source x - e_i lies
 * beyond (bit a set for axis a), with the kinds found there: *bb = 1 if one of
 * them is BOUNCEBACK, *nf = mask of the NOFLUX_NODE ones. */
static int beyond(const orc_lattice* L, const orc_params* p, int i, int64_t x, int64_t y, int64_t z, int* bb,
                  int* nf)
{
    const int64_t c[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
    int mask = 0;
    *bb = 0;
    *nf = 0;
    for (int a = 0; a < 3; ++a) {
        const int e = L->e[i][a];
        if (e == 0) continue;
        const int side = e > 0 ? 0 : 1;   /* e > 0: the source lies below the low face */
        const int kind = face_kind(p, a, side);
        if (kind == ORC_PERIODIC) continue;
        if ((e > 0 && c[a] == 0) || (e < 0 && c[a] == n[a] - 1)) {
            mask |= 1 << a;
            if (kind == ORC_BOUNCEBACK) *bb = 1;
            if (kind == ORC_NOFLUX_NODE) *nf |= 1 << a;
        }
    }
    return mask;
}

static void set_threads(const orc_params* p)
{
#ifdef _OPENMP
    if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#else
    (void)p;
#endif
}

/* ---------------------------------------------------------------------- */
/* Public entry points                                                     */
/* ---------------------------------------------------------------------- */

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Copies out the lattice tables the oracle uses (for the pins). */
int orc_lattice_tables(const orc_params* p, int* e_out, double* M_out, double* Minv_out,
                       double* S_out)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    for (int i = 0; i < L.q; ++i)
        for (int a = 0; a < 3; ++a) e_out[i * 3 + a] = L.e[i][a];
    for (int r = 0; r < L.q; ++r)
        for (int c = 0; c < L.q; ++c) {
            M_out[r * L.q + c] = L.M[r][c];
            Minv_out[r * L.q + c] = L.Minv[r][c];
            S_out[r * L.q + c] = L.S[r][c];
        }
    return 0;
}

/* Equilibrium moments at one node (for the pins). */
int orc_meq(const orc_params* p, double phi, const double* u, double* m_out)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    double uu[3] = {u[0], u[1], L.dim == 3 ? u[2] : 0.0};
    meq(&L, p, phi, uu, m_out);
    return 0;
}

/* One collision at one node (for the pins). */
int orc_collide_node(const orc_params* p, const double* f, const double* u, double* fout)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    double uu[3] = {u[0], u[1], L.dim == 3 ? u[2] : 0.0};
    collide_node(&L, p, f, uu, fout);
    return 0;
}

/* f^eq = M^-1 m^eq(phi, u) in every cell (the initial state). */
int orc_init_eq(const orc_params* p, const double* phi, const double* u, double* f)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    const int64_t nc = ncells(p);
    set_threads(p);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        double uu[3], me[ORC_MAXQ], fe[ORC_MAXQ];
        get_u(&L, u, nc, c, uu);
        meq(&L, p, phi[c], uu, me);
        matvec(L.q, L.Minv, me, fe);
        for (int i = 0; i < L.q; ++i) f[i * nc + c] = fe[i];
    }
    return 0;
}

/* phi = sum_i f_i (Eq. 8). */
int orc_phi(const orc_params* p, const double* f, double* phi)
{
    const int64_t nc = ncells(p);
    set_threads(p);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        double s = 0.0;
        for (int i = 0; i < p->q; ++i) s += f[i * nc + c];
        phi[c] = s;
    }
    return 0;
}

/* Wall rules at the wall nodes, after streaming (and after the bounce-back of
 * the push):
 *   NOFLUX_NODE: the Neumann rule of Sec. 3.2 (bottom f2=f4, f5=f8, f6=f7;
 *                top f4=f2, f7=f6, f8=f5): a population whose source lies beyond
 *                Neumann walls copies the population reflected in the axes of
 *                those walls (on the y faces alone: its mirror image in y; at an
 *                edge of two Neumann faces, the population reflected in both).
 *   DIRICHLET:   (y faces only) every population whose source lies beyond the
 *                wall is set to f^eq_i(phi*, u) with phi* chosen so that
 *                sum_i f_i = phi_w.
 *   BOUNCEBACK is applied during the push itself. */
static void wall_fill(const orc_lattice* L, const orc_params* p, const double* u, double* fn)
{
    const int64_t nx = p->nx, ny = p->ny, nz = p->nz, nc = ncells(p);
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                if (!on_wall(p, x, y, z)) continue;
                const int64_t c = x + nx * (y + ny * z);
                double v[ORC_MAXQ];
                for (int i = 0; i < L->q; ++i) v[i] = fn[i * nc + c];
                for (int i = 0; i < L->q; ++i) {
                    int bb, nf;
                    beyond(L, p, i, x, y, z, &bb, &nf);
                    if (nf) fn[i * nc + c] = v[reflect(L, i, nf)];
                }
            }
    for (int side = 0; side < 2; ++side) {
        const int kind = side == 0 ? p->bc_lo : p->bc_hi;
        if (kind != ORC_DIRICHLET) continue;
        const int64_t y = side == 0 ? 0 : ny - 1;
        const int inward = side == 0 ? +1 : -1; /* e_y of the unknown populations */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t c = x + nx * (y + ny * z);
                double uu[3], me[ORC_MAXQ], w[ORC_MAXQ];
                get_u(L, u, nc, c, uu);
                meq(L, p, 1.0, uu, me);
                matvec(L->q, L->Minv, me, w); /* f^eq at unit phi */
                double known = 0.0, wk = 0.0;
                for (int i = 0; i < L->q; ++i) {
                    if (L->e[i][1] == inward) wk += w[i];
                    else known += fn[i * nc + c];
                }
                const double phiw = side == 0 ? p->phi_w_lo : p->phi_w_hi;
                const double phis = (phiw - known) / wk;
                for (int i = 0; i < L->q; ++i)
                    if (L->e[i][1] == inward) fn[i * nc + c] = phis * w[i];
            }
    }
}

/* One time step, f(t) -> f(t+1): collide every node with u(x, t) (Eq. 13 with
 * Eq. 31 / 24 / A.5), push-stream (Eq. 5), then the wall rules.  fpost is a
 * caller-provided scratch array of q*ncell doubles; f_out must not alias f_in. */
int orc_step(const orc_params* p, const double* f_in, const double* u, double* fpost,
             double* f_out)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    const int64_t nx = p->nx, ny = p->ny, nz = p->nz, nc = ncells(p);
    const int q = L.q;
    set_threads(p);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        double fl[ORC_MAXQ], fo[ORC_MAXQ], uu[3];
        for (int i = 0; i < q; ++i) fl[i] = f_in[i * nc + c];
        get_u(&L, u, nc, c, uu);
        collide_node(&L, p, fl, uu, fo);
        for (int i = 0; i < q; ++i) fpost[i * nc + c] = fo[i];
    }
    for (int64_t k = 0; k < (int64_t)q * nc; ++k) f_out[k] = 0.0;
    const int per[3] = {p->bcx_lo == ORC_PERIODIC, p->bc_lo == ORC_PERIODIC, p->bcz_lo == ORC_PERIODIC};
    const int64_t n[3] = {nx, ny, nz};
    int opp[ORC_MAXQ];
    for (int i = 0; i < q; ++i) opp[i] = opposite(&L, i);
    /* Eq. 5: f_i(x + e_i, t + 1) = f'_i(x, t).  Parallel over destination
     * planes i: each plane is written by exactly one thread; populations that
     * would leave through a wall are left to the serial pass below. */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < q; ++i) {
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c = x + nx * (y + ny * z);
                    const int64_t r[3] = {x, y, z};
                    int64_t d[3];
                    int out = 0;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = r[a] + L.e[i][a];
                        if (per[a]) d[a] = wrap(d[a], n[a]);
                        else if (d[a] < 0 || d[a] >= n[a]) out = 1; /* leaves through a wall */
                    }
                    if (out) continue;
                    f_out[i * nc + d[0] + nx * (d[1] + ny * d[2])] = fpost[i * nc + c];
                }
    }
    if (any_wall(p)) {
        /* Halfway bounce-back: a population that would leave through a wall of
         * which (one) is BOUNCEBACK returns to its node in the opposite
         * direction; the population opp(i) there has its source beyond the same
         * faces, so nothing else writes it. */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    if (!on_wall(p, x, y, z)) continue;
                    const int64_t c = x + nx * (y + ny * z);
                    for (int i = 0; i < q; ++i) {
                        int bb, nf;
                        if (beyond(&L, p, opp[i], x, y, z, &bb, &nf) && bb)
                            f_out[opp[i] * nc + c] = fpost[i * nc + c];
                    }
                }
        wall_fill(&L, p, u, f_out);
    }
    return 0;
}

/* Runs nsteps with a velocity that is constant in time (u may be NULL). */
int orc_run(const orc_params* p, double* f, const double* u, int64_t nsteps)
{
    const int64_t n = (int64_t)p->q * ncells(p);
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    if (!a || !b) { free(a); free(b); return -10; }
    int rc = 0;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_step(p, f, u, a, b);
        memcpy(f, b, sizeof(double) * n);
    }
    free(a);
    free(b);
    return rc;
}

/* Explicit collision matrix C(u) = M^-1 [I - S (I - J)] M with
 * J = d m^eq / d m = (m^eq at unit phi) e_0^T: the step is linear in f for
 * a fixed u (Eq. 11-15). */
static void collision_matrix(const orc_lattice* L, const orc_params* p, const double u[3],
                             double C[ORC_MAXQ][ORC_MAXQ])
{
    const int q = L->q;
    double v[ORC_MAXQ], K[ORC_MAXQ][ORC_MAXQ], T[ORC_MAXQ][ORC_MAXQ];
    meq(L, p, 1.0, u, v);
    for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) {
            /* (I - J)[k][c] = delta_kc - v_k delta_c0 ;  K = I - S (I - J) */
            double acc = 0.0;
            for (int k = 0; k < q; ++k) {
                const double imj = (k == c ? 1.0 : 0.0) - (c == 0 ? v[k] : 0.0);
                acc += L->S[r][k] * imj;
            }
            K[r][c] = (r == c ? 1.0 : 0.0) - acc;
        }
    for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) {
            double acc = 0.0;
            for (int k = 0; k < q; ++k) acc += K[r][k] * L->M[k][c];
            T[r][c] = acc;
        }
    for (int r = 0; r < q; ++r)
        for (int c = 0; c < q; ++c) {
            double acc = 0.0;
            for (int k = 0; k < q; ++k) acc += L->Minv[r][k] * T[k][c];
            C[r][c] = acc;
        }
}

/* Reverse-time (adjoint) step of orc_step for a fixed velocity field.
 *   lam_next : adjoint of f(t+1)            [q*ncell]
 *   f_pre    : the forward state f(t)       [q*ncell]
 *   u        : the velocity used at time t  [dim*ncell] or NULL
 *   lam_out  : adjoint of f(t)              [q*ncell]
 *   dS       : += dL/dS_kl summed over cells [q*q] (or NULL)
 *   du       : += dL/du_a(x, t)             [dim*ncell] (or NULL)
 * The streaming part is the literal transpose of the push + wall rules in
 * orc_step (walls on any face), applied in reverse order; the collision part
 * multiplies by C^T. A Dirichlet wall makes the step affine; its linear part is
 * transposed, and velocity partials (du) are not formed with one (-4). */
int orc_adjoint_step(const orc_params* p, const double* lam_next, const double* f_pre,
                     const double* u, double* lam_out, double* dS, double* du)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    /* Dirichlet walls: the fill is affine in f; its linear part is transposed below.
     * Velocity partials through the fill (its weights depend on u) are not formed. */
    if ((p->bc_lo == ORC_DIRICHLET || p->bc_hi == ORC_DIRICHLET) && du) return -4;
    const int64_t nx = p->nx, ny = p->ny, nz = p->nz, nc = ncells(p);
    const int q = L.q;
    double* lam = (double*)malloc(sizeof(double) * q * nc);  /* adjoint of f(t+1) before wall fill */
    double* lpost = (double*)calloc((size_t)q * nc, sizeof(double)); /* adjoint of f'(t) */
    if (!lam || !lpost) { free(lam); free(lpost); return -10; }
    memcpy(lam, lam_next, sizeof(double) * q * nc);
    int opp[ORC_MAXQ];
    for (int i = 0; i < q; ++i) opp[i] = opposite(&L, i);
    if (any_wall(p)) {
        /* transpose of the Dirichlet fill (the last rule of wall_fill): at a wall node
         * of a DIRICHLET face the inward populations are f_i = phi_s w_i with
         * w = f^eq(1, u), W = sum of the inward w_i and phi_s = (phi_w - sum of the
         * other populations) / W, so each other population j receives
         * -sum_i w_i lam_i / W and the inward ones carry nothing further back */
        for (int side = 0; side < 2; ++side) {
            const int kind = side == 0 ? p->bc_lo : p->bc_hi;
            if (kind != ORC_DIRICHLET) continue;
            const int64_t y = side == 0 ? 0 : ny - 1;
            const int inward = side == 0 ? +1 : -1;
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c = x + nx * (y + ny * z);
                    double uu[3], me[ORC_MAXQ], w[ORC_MAXQ];
                    get_u(&L, u, nc, c, uu);
                    meq(&L, p, 1.0, uu, me);
                    matvec(q, L.Minv, me, w);
                    double W = 0.0, lw = 0.0;
                    for (int i = 0; i < q; ++i)
                        if (L.e[i][1] == inward) {
                            W += w[i];
                            lw += w[i] * lam[i * nc + c];
                        }
                    for (int i = 0; i < q; ++i) {
                        if (L.e[i][1] == inward) lam[i * nc + c] = 0.0;
                        else lam[i * nc + c] -= lw / W;
                    }
                }
        }
        /* transpose of the NOFLUX_NODE fill of wall_fill: at a wall node the
         * populations whose source lies beyond NOFLUX_NODE faces took the value
         * (before the fill) of the population reflected in those axes */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    if (!on_wall(p, x, y, z)) continue;
                    const int64_t c = x + nx * (y + ny * z);
                    double acc[ORC_MAXQ] = {0.0};
                    for (int i = 0; i < q; ++i) {
                        int bb, nf;
                        beyond(&L, p, i, x, y, z, &bb, &nf);
                        acc[nf ? reflect(&L, i, nf) : i] += lam[i * nc + c];
                    }
                    for (int i = 0; i < q; ++i) lam[i * nc + c] = acc[i];
                }
        /* transpose of bounce-back: f_opp(i)(x) = f'_i(x) where the source of
         * opp(i) lies beyond a BOUNCEBACK face */
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    if (!on_wall(p, x, y, z)) continue;
                    const int64_t c = x + nx * (y + ny * z);
                    for (int i = 0; i < q; ++i) {
                        int bb, nf;
                        if (beyond(&L, p, opp[i], x, y, z, &bb, &nf) && bb) lpost[i * nc + c] += lam[opp[i] * nc + c];
                    }
                }
    }
    /* transpose of the push (Eq. 5): populations that leave through a wall carry nothing */
    const int per[3] = {p->bcx_lo == ORC_PERIODIC, p->bc_lo == ORC_PERIODIC, p->bcz_lo == ORC_PERIODIC};
    const int64_t n[3] = {nx, ny, nz};
    for (int i = 0; i < q; ++i)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c = x + nx * (y + ny * z);
                    const int64_t r[3] = {x, y, z};
                    int64_t d[3];
                    int out = 0;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = r[a] + L.e[i][a];
                        if (per[a]) d[a] = wrap(d[a], n[a]);
                        else if (d[a] < 0 || d[a] >= n[a]) out = 1;
                    }
                    if (out) continue;
                    lpost[i * nc + c] += lam[i * nc + d[0] + nx * (d[1] + ny * d[2])];
                }
    /* transpose of the collision: lam(t) = C^T lam'(t) ; parameter and velocity partials */
    set_threads(p);
    double* dS_thread = NULL;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    if (dS) dS_thread = (double*)calloc((size_t)nthr * q * q, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double uu[3], C[ORC_MAXQ][ORC_MAXQ], lp[ORC_MAXQ], lo[ORC_MAXQ];
        get_u(&L, u, nc, c, uu);
        collision_matrix(&L, p, uu, C);
        for (int i = 0; i < q; ++i) lp[i] = lpost[i * nc + c];
        matTvec(q, C, lp, lo);
        for (int i = 0; i < q; ++i) lam_out[i * nc + c] = lo[i];
        if (dS || du) {
            double fl[ORC_MAXQ], m[ORC_MAXQ], me[ORC_MAXQ], mu[ORC_MAXQ];
            for (int i = 0; i < q; ++i) fl[i] = f_pre[i * nc + c];
            matvec(q, L.M, fl, m);
            meq(&L, p, m[0], uu, me);
            matTvec(q, L.Minv, lp, mu); /* mu = M^-T lam' */
            if (dS_thread) {
                /* f' = M^-1 (m - S (m - m^eq))  =>  dL/dS_kl = -mu_k (m - m^eq)_l */
                double* acc = dS_thread + (size_t)tid * q * q;
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l) acc[k * q + l] -= mu[k] * (m[l] - me[l]);
            }
            if (du) {
                /* df'/du_a = M^-1 S phi dm^eq/du_a */
                for (int a = 0; a < L.dim; ++a) {
                    double d[ORC_MAXQ], sd[ORC_MAXQ];
                    dmeq_du(&L, p, uu, a, d);
                    for (int k = 0; k < q; ++k) d[k] *= m[0];
                    matvec(q, L.S, d, sd);
                    double g = 0.0;
                    for (int k = 0; k < q; ++k) g += mu[k] * sd[k];
                    du[a * nc + c] += g;
                }
            }
        }
    }
    if (dS_thread) {
        for (int t = 0; t < nthr; ++t)
            for (int k = 0; k < q * q; ++k) dS[k] += dS_thread[(size_t)t * q * q + k];
        free(dS_thread);
    }
    free(lam);
    free(lpost);
    return 0;
}

/* d f^eq_i / d phi and d f^eq_i / d u_a at every cell (for the gradient of
 * the initial state f(0) = f^eq(phi_0, u(0))).  dfeq_dphi: [q*ncell];
 * dfeq_du: [dim*q*ncell] (may be NULL). */
int orc_feq_jacobian(const orc_params* p, const double* phi, const double* u, double* dfeq_dphi,
                     double* dfeq_du)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    const int64_t nc = ncells(p);
    for (int64_t c = 0; c < nc; ++c) {
        double uu[3], me[ORC_MAXQ], fe[ORC_MAXQ];
        get_u(&L, u, nc, c, uu);
        meq(&L, p, 1.0, uu, me);
        matvec(L.q, L.Minv, me, fe);
        for (int i = 0; i < L.q; ++i) dfeq_dphi[i * nc + c] = fe[i];
        if (dfeq_du) {
            for (int a = 0; a < L.dim; ++a) {
                double d[ORC_MAXQ], fd[ORC_MAXQ];
                dmeq_du(&L, p, uu, a, d);
                matvec(L.q, L.Minv, d, fd);
                for (int i = 0; i < L.q; ++i)
                    dfeq_du[((size_t)a * L.q + i) * nc + c] = phi[c] * fd[i];
            }
        }
    }
    return 0;
}

/* Exact spatial-moment recursion for a channel that is uniform and unbounded
 * in x (Taylor-Aris set-up of Sec. 3.2).  Because the collision is linear in f
 * with coefficients that depend on y only, the moments
 *     F^k_i(y) = sum_x x^k f_i(x, y),  k = 0, 1, 2,
 * evolve in closed form: collision acts on each F^k(y) like on f, and the push
 * f_i(x + e_ix, y + e_iy) = f'_i(x, y) maps F'^k_i(y) to
 *     sum_j binom(k, j) e_ix^(k-j) F'^j_i(y)  at row y + e_iy;
 * the wall rules copy whole rows and so act identically on every F^k.
 * This is the same arithmetic as orc_step applied to an unbounded x axis.
 *
 *   ux_row : u_x at the ny nodes (u_y = 0)
 *   F0     : [3*q*ny] initial moments (k-major, then i, then y)
 *   wy     : [ny] cross-section weights used for phi-bar
 *   out    : [nsteps+1][3] = sum_y wy * sum_i F^k_i(y) for k = 0, 1, 2
 *            (out[0] is the initial state). */
int orc_channel_moments(const orc_params* p, const double* ux_row, const double* F0,
                        const double* wy, int64_t nsteps, double* out)
{
    orc_lattice L;
    int rc = build_lattice(&L, p);
    if (rc) return rc;
    if (L.q != 9) return -5;
    const int q = 9;
    const int64_t ny = p->ny;
    const int periodic_y = (p->bc_lo == ORC_PERIODIC);
    const size_t nF = (size_t)3 * q * ny;
    double* F = (double*)malloc(sizeof(double) * nF);
    double* Fp = (double*)malloc(sizeof(double) * nF);
    double* Fn = (double*)malloc(sizeof(double) * nF);
    if (!F || !Fp || !Fn) { free(F); free(Fp); free(Fn); return -10; }
    memcpy(F, F0, sizeof(double) * nF);
    int opp[ORC_MAXQ];
    for (int i = 0; i < q; ++i) opp[i] = opposite(&L, i);
    /* u depends on y only and is steady, so each row's collision matrix is
     * built once */
    double (*Crow)[ORC_MAXQ][ORC_MAXQ] = malloc(sizeof(double) * ORC_MAXQ * ORC_MAXQ * ny);
    if (!Crow) { free(F); free(Fp); free(Fn); return -10; }
    for (int64_t y = 0; y < ny; ++y) {
        double uu[3] = {ux_row[y], 0.0, 0.0};
        collision_matrix(&L, p, uu, Crow[y]);
    }
#define FK(arr, k, i, y) (arr)[((size_t)(k) * q + (i)) * ny + (y)]
    for (int64_t s = 0; s <= nsteps; ++s) {
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int64_t y = 0; y < ny; ++y) {
                double r = 0.0;
                for (int i = 0; i < q; ++i) r += FK(F, k, i, y);
                acc += wy[y] * r;
            }
            out[s * 3 + k] = acc;
        }
        if (s == nsteps) break;
        /* collision: linear in f, so the k = 1, 2 moments are collided with
         * the same matrix but without the inhomogeneous part; C(u) covers
         * both since m^eq is linear in phi. */
        for (int64_t y = 0; y < ny; ++y) {
            for (int k = 0; k < 3; ++k) {
                double v[ORC_MAXQ], w[ORC_MAXQ];
                for (int i = 0; i < q; ++i) v[i] = FK(F, k, i, y);
                matvec(q, (const double(*)[ORC_MAXQ])Crow[y], v, w);
                for (int i = 0; i < q; ++i) FK(Fp, k, i, y) = w[i];
            }
        }
        memset(Fn, 0, sizeof(double) * nF);
        for (int i = 0; i < q; ++i) {
            const double ex = L.e[i][0];
            for (int64_t y = 0; y < ny; ++y) {
                int64_t yd = y + L.e[i][1];
                if (periodic_y) yd = wrap(yd, ny);
                else if (yd < 0 || yd >= ny) {
                    int kind = (yd < 0) ? p->bc_lo : p->bc_hi;
                    if (kind == ORC_BOUNCEBACK) {
                        /* returns to (x, y) in direction opp(i): no x shift */
                        for (int k = 0; k < 3; ++k) FK(Fn, k, opp[i], y) += FK(Fp, k, i, y);
                    }
                    continue;
                }
                const double f0 = FK(Fp, 0, i, y), f1 = FK(Fp, 1, i, y), f2 = FK(Fp, 2, i, y);
                FK(Fn, 0, i, yd) += f0;
                FK(Fn, 1, i, yd) += f1 + ex * f0;
                FK(Fn, 2, i, yd) += f2 + 2.0 * ex * f1 + ex * ex * f0;
            }
        }
        if (!periodic_y) {
            for (int side = 0; side < 2; ++side) {
                const int kind = side == 0 ? p->bc_lo : p->bc_hi;
                if (kind != ORC_NOFLUX_NODE) continue;
                const int64_t y = side == 0 ? 0 : ny - 1;
                const int inward = side == 0 ? +1 : -1;
                for (int i = 0; i < q; ++i)
                    if (L.e[i][1] == inward)
                        for (int k = 0; k < 3; ++k) FK(Fn, k, i, y) = FK(Fn, k, mirror_y(&L, i), y);
            }
        }
        double* t = F; F = Fn; Fn = t;
    }
#undef FK
    free(Crow);
    free(F);
    free(Fp);
    free(Fn);
    return 0;
}
