/*
 * FP64 CPU oracle for the lattice Boltzmann method for the volume-averaged
 * Navier-Stokes equations (VANSE) with Carreau-Yasuda rheology of
 * Horvat, Lunowa, Sytnyk, Wohlmuth, "A Lattice Boltzmann Method for
 * Non-Newtonian Blood Flow in Coiled Intracranial Aneurysms" (arXiv 2402.10809).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it; the library path never does.  It
 * shares no code, table or constant with the CUDA path.
 *
 * It follows the paper literally, in the paper's push form (Sec. 3, collision
 * then streaming):
 *   f_i(t+1, x+c_i) = f_i(t,x) + Omega^phi_i + Omega^f_i + Omega^SRT_i,
 * all arithmetic in double precision, one fluid cell at a time.
 *
 * State convention: f holds the pre-collision populations f(t) of every fluid
 * cell after streaming, bounce-back and the inlet/outlet reconstruction of
 * time t; omega holds the relaxation rate of the last collision, omega(t-1).
 * Readings of points the paper leaves open are marked READING.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OQMAX 27
#define CS2 (1.0 / 3.0)

enum { O_SOLID = 0, O_FLUID = 1, O_INLET = 2, O_OUTLET = 3 };

typedef struct {
    int32_t nx, ny, nz, q;
    int32_t periodic[3];
    /* Carreau-Yasuda parameters (SI) and the lattice scales of Table 1. */
    double mu0, mu_inf, lam, n_cy, a_cy, rho0, dx, dt;
    /* Porous closure (SI): grain size d_p, optional constant permeability
     * k_const (> 0 overrides Kozeny-Carman), Darcy viscosity nu_darcy (<= 0:
     * nu = mu0 / rho0 as in Sec. 4), Forchheimer term on/off. */
    double d_p, k_const, nu_darcy;
    int32_t forchheimer;
    double g[3];              /* body force per unit mass, lattice units */
    int32_t in_axis, in_side; /* in_axis < 0: no inlet */
    double in_center[3], in_radius, u0, amp, period, ramp;
    int32_t out_axis, out_side; /* out_axis < 0: no outlet */
    double rho_out;
} oracle_params;

typedef struct {
    oracle_params p;
    /* lattice units */
    double mu0, mu_inf, lam, nu_d, d_p, k_const;
    int q;
    int c[OQMAX][3];
    double w[OQMAX];
    int opp[OQMAX];
    int64_t n_box, nf;
    uint8_t* flags;
    double* phi;
    int64_t* cell;   /* [nf] dense index of each fluid cell */
    int64_t* slot;   /* [n_box] position in the fluid list, -1 for solid */
    double* f;       /* [nf][q] pre-collision populations f(t) */
    double* fpost;   /* [nf][q] post-collision populations */
    double* fnew;    /* [nf][q] streaming target */
    double* omega;   /* [nf] omega(t-1) */
    double* omega_new;
    double* aniso_s;      /* [n_box][6] shape tensor S (xx yy zz xy xz yz), or NULL */
    double* aniso_s_half; /* [n_box][6] its square root S^{1/2} */
    int64_t t;
} oracle_ctx;

/* ---------------------------------------------------------------- lattice */

/* D3Q27 (the paper's choice, Sec. 3) or D3Q19, c_s^2 = 1/3.  The paper defers
 * the weights to the textbooks; they are the standard values by |c|^2:
 * D3Q27 8/27, 2/27, 1/54, 1/216; D3Q19 1/3, 1/18, 1/36. */
static int lattice_build(oracle_ctx* o)
{
    int q = o->p.q, n = 0;
    if (q != 19 && q != 27) return -1;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int k = cx * cx + cy * cy + cz * cz;
                if (q == 19 && k == 3) continue;
                o->c[n][0] = cx; o->c[n][1] = cy; o->c[n][2] = cz;
                if (q == 27) o->w[n] = k == 0 ? 8.0 / 27 : k == 1 ? 2.0 / 27 : k == 2 ? 1.0 / 54 : 1.0 / 216;
                else         o->w[n] = k == 0 ? 1.0 / 3 : k == 1 ? 1.0 / 18 : 1.0 / 36;
                ++n;
            }
    o->q = n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (o->c[j][0] == -o->c[i][0] && o->c[j][1] == -o->c[i][1] && o->c[j][2] == -o->c[i][2])
                o->opp[i] = j;
    return 0;
}

/* ------------------------------------------------------------ geometry */

static void coords(const oracle_ctx* o, int64_t idx, int* x, int* y, int* z)
{
    *x = (int)(idx % o->p.nx);
    *y = (int)((idx / o->p.nx) % o->p.ny);
    *z = (int)(idx / ((int64_t)o->p.nx * o->p.ny));
}

/* Dense index of (x,y,z)+d with periodic wrap.  Returns -1 when the target
 * leaves the box across a non-periodic face; *axis / *side name that face. */
static int64_t neighbour(const oracle_ctx* o, int x, int y, int z, const int d[3], int* axis, int* side)
{
    int v[3] = {x + d[0], y + d[1], z + d[2]};
    int n[3] = {o->p.nx, o->p.ny, o->p.nz};
    *axis = -1; *side = 0;
    for (int a = 0; a < 3; ++a) {
        if (v[a] < 0 || v[a] >= n[a]) {
            if (o->p.periodic[a]) {
                v[a] = (v[a] + n[a]) % n[a];
            } else {
                *axis = a; *side = v[a] < 0 ? 0 : 1;
                return -1;
            }
        }
    }
    return v[0] + (int64_t)n[0] * (v[1] + (int64_t)n[1] * v[2]);
}

/* ------------------------------------------------------ local physics */

/* Kozeny-Carman permeability and Ergun's Forchheimer constant (Sec. 2):
 * k = phi^3 d_p^2 / (150 (1-phi)^2), C_F = 1.75 / sqrt(150 phi^3).
 * Returns 1/k and 1/sqrt(k); both vanish at phi = 1 (k infinite: pure fluid). */
static void porous_closure(const oracle_ctx* o, double phi, double* inv_k, double* inv_sqrt_k, double* cf)
{
    if (o->k_const > 0.0) {
        /* READING: a constant permeability acts only where there is solid. */
        *inv_k = phi < 1.0 ? 1.0 / o->k_const : 0.0;
        *inv_sqrt_k = phi < 1.0 ? 1.0 / sqrt(o->k_const) : 0.0;
    } else {
        double k = phi * phi * phi * o->d_p * o->d_p / (150.0 * (1.0 - phi) * (1.0 - phi));
        *inv_k = 1.0 / k;          /* k = +inf at phi = 1 gives 0 */
        *inv_sqrt_k = 1.0 / sqrt(k);
    }
    *cf = o->p.forchheimer ? 1.75 / sqrt(150.0 * phi * phi * phi) : 0.0;
}

/* Solves X x = b for a 3x3 matrix by Gaussian elimination with partial
 * pivoting. */
static void solve3(const double Xin[3][3], const double b[3], double x[3])
{
    double X[3][4];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) X[r][c] = Xin[r][c];
        X[r][3] = b[r];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(X[r][c]) > fabs(X[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 4; ++k) { double t = X[c][k]; X[c][k] = X[piv][k]; X[piv][k] = t; }
        for (int r = c + 1; r < 3; ++r) {
            double m = X[r][c] / X[c][c];
            for (int k = c; k < 4; ++k) X[r][k] -= m * X[c][k];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double acc = X[r][3];
        for (int k = r + 1; k < 3; ++k) acc -= X[r][k] * x[k];
        x[r] = acc / X[r][r];
    }
}

/* Symmetric 3x3 matrix from its six components xx yy zz xy xz yz. */
static void sym3(const double* s, double M[3][3])
{
    M[0][0] = s[0]; M[1][1] = s[1]; M[2][2] = s[2];
    M[0][1] = M[1][0] = s[3];
    M[0][2] = M[2][0] = s[4];
    M[1][2] = M[2][1] = s[5];
}

/* Anisotropic permeability (Sec. 3, remark on the velocity solution): the drag
 * f(u) = -phi^2 nu K^{-1} u - phi^3 C_F |u| K^{-1/2} u makes the velocity
 * equation (A + |u| B) u = v, A = Id + (phi nu dt / 2) K^{-1},
 * B = (phi^2 C_F dt / 2) K^{-1/2}, which the paper solves by the fixed-point
 * iteration u_{m+1} = X_m^{-1} v, X_m = A + |u_m| B.
 * READING: K = k(phi) S^{-1} with the isotropic closure k(phi) of
 * porous_closure and a dimensionless SPD shape tensor S per cell, so that
 * K^{-1} = S / k and K^{-1/2} = S^{1/2} / sqrt(k); C_F stays Ergun's scalar.
 * READING: u_0 = v (no extra state); the iteration runs until
 * |u_{m+1} - u_m| <= 1e-15 |v|, at most 200 times.  Returns F = rho (g + f(u)). */
static void anisotropic_velocity(const oracle_ctx* o, int64_t idx, double phi, double rho, const double v[3],
                                 double u[3], double F[3])
{
    double inv_k, inv_sqrt_k, cf;
    porous_closure(o, phi, &inv_k, &inv_sqrt_k, &cf);
    double S[3][3], Sh[3][3], Kinv[3][3], Kinvh[3][3], A[3][3], B[3][3];
    sym3(o->aniso_s + idx * 6, S);
    sym3(o->aniso_s_half + idx * 6, Sh);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Kinv[a][b] = S[a][b] * inv_k;
            Kinvh[a][b] = Sh[a][b] * inv_sqrt_k;
            A[a][b] = (a == b ? 1.0 : 0.0) + phi * o->nu_d / 2.0 * Kinv[a][b];
            B[a][b] = phi * phi * cf / 2.0 * Kinvh[a][b];
        }
    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) u[a] = v[a];
    for (int m = 0; m < 200; ++m) {
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double X[3][3], un1[3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) X[a][b] = A[a][b] + un * B[a][b];
        solve3(X, v, un1);
        double d = 0.0;
        for (int a = 0; a < 3; ++a) { d += (un1[a] - u[a]) * (un1[a] - u[a]); u[a] = un1[a]; }
        if (sqrt(d) <= 1e-15 * vn) break;
    }
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) {
        double fd = 0.0;
        for (int b = 0; b < 3; ++b)
            fd -= phi * phi * o->nu_d * Kinv[a][b] * u[b] + phi * phi * phi * cf * un * Kinvh[a][b] * u[b];
        F[a] = rho * (o->p.g[a] + fd);
    }
}

/* Macroscopic quantities (Sec. 3):
 *   rho = phi^{-1} sum_i f_i,
 *   u   = (phi rho)^{-1} (sum_i f_i c_i + rho f(u) / 2),
 * solved explicitly with the preliminary velocity v:
 *   u = v / (C0 + sqrt(C0^2 + C1 |v|)),  C0 = 1/2 + phi nu / (4k),
 *   C1 = phi^2 C_F / (2 sqrt(k))     (dt = 1).
 * READING: a body force g (per unit mass) adds to the drag, f = g + f_d(u);
 * solving the same quadratic with v = (sum f c + rho g / 2) / (phi rho).
 * Returns F = rho (g + f_d(u)), f_d = -phi^2 nu u / k - phi^3 C_F |u| u / sqrt(k). */
static void macroscopic(const oracle_ctx* o, const double* f, int64_t idx, double* rho_out,
                        double u[3], double F[3])
{
    double phi = o->phi[idx];
    double s = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < o->q; ++i) {
        s += f[i];
        for (int a = 0; a < 3; ++a) m[a] += f[i] * o->c[i][a];
    }
    double rho = s / phi;
    double v[3], vn = 0.0;
    for (int a = 0; a < 3; ++a) {
        v[a] = (m[a] + 0.5 * rho * o->p.g[a]) / (phi * rho);
        vn += v[a] * v[a];
    }
    vn = sqrt(vn);
    if (o->aniso_s && phi < 1.0) {
        /* READING: the tensor acts where there is solid (phi < 1), like the
         * constant permeability; pure fluid has no drag. */
        anisotropic_velocity(o, idx, phi, rho, v, u, F);
        *rho_out = rho;
        return;
    }
    double inv_k, inv_sqrt_k, cf;
    porous_closure(o, phi, &inv_k, &inv_sqrt_k, &cf);
    double c0 = 0.5 + phi * o->nu_d * inv_k / 4.0;
    double c1 = phi * phi * cf * inv_sqrt_k / 2.0;
    double den = c0 + sqrt(c0 * c0 + c1 * vn);
    double un = 0.0;
    for (int a = 0; a < 3; ++a) { u[a] = v[a] / den; un += u[a] * u[a]; }
    un = sqrt(un);
    for (int a = 0; a < 3; ++a) {
        double fd = -phi * phi * o->nu_d * inv_k * u[a] - phi * phi * phi * cf * inv_sqrt_k * un * u[a];
        F[a] = rho * (o->p.g[a] + fd);
    }
    *rho_out = rho;
}

/* Porosity-weighted equilibrium (Sec. 3):
 * f_i^eq = w_i phi rho (1 + c_i.u / c_s^2 + (c_i.u)^2 / (2 c_s^4) - u.u / (2 c_s^2)). */
static double equilibrium(const oracle_ctx* o, int i, double phi, double rho, const double u[3])
{
    double cu = o->c[i][0] * u[0] + o->c[i][1] * u[1] + o->c[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return o->w[i] * phi * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Carreau-Yasuda law, Eq. (3):
 * mu = mu_inf + (mu0 - mu_inf) (1 + (lambda gdot)^a)^((n-1)/a). */
static double carreau_yasuda(const oracle_ctx* o, double gdot)
{
    return o->mu_inf + (o->mu0 - o->mu_inf) * pow(1.0 + pow(o->lam * gdot, o->p.a_cy), (o->p.n_cy - 1.0) / o->p.a_cy);
}

/* Relaxation rate from the dynamic viscosity (Sec. 3):
 * omega = 2 rho c_s^2 dt (2 mu + rho c_s^2 dt)^{-1}. */
static double omega_of(double rho, double mu)
{
    return 2.0 * rho * CS2 / (2.0 * mu + rho * CS2);
}

/* Corrected second moment and shear rate (Sec. 3):
 *   Pi = sum_i (f_i - f_i^eq) c_i (x) c_i + (rho f (x) u + u (x) rho f) / 2,
 *   gdot(t) = omega(t-1) ||Pi||_F / (c_s^2 rho). */
static double shear_rate(const oracle_ctx* o, const double* f, double phi, double rho, const double u[3],
                         const double F[3], double omega_prev)
{
    double pi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) pi[a][b] = 0.5 * (F[a] * u[b] + u[a] * F[b]);
    for (int i = 0; i < o->q; ++i) {
        double d = f[i] - equilibrium(o, i, phi, rho, u);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) pi[a][b] += d * o->c[i][a] * o->c[i][b];
    }
    double nrm = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) nrm += pi[a][b] * pi[a][b];
    return omega_prev * sqrt(nrm) / (CS2 * rho);
}

/* Porosity seen across link i of cell (x,y,z).  READING: where the neighbour is
 * solid or outside the box, it takes the cell's own porosity, so that
 * Omega^phi_i vanishes on that link. */
static double link_porosity(const oracle_ctx* o, int x, int y, int z, int i, double phi_self)
{
    int ax, sd;
    int64_t d = neighbour(o, x, y, z, o->c[i], &ax, &sd);
    if (d < 0 || o->flags[d] == O_SOLID) return phi_self;
    return o->phi[d];
}

/* One collision (Sec. 3): returns the post-collision populations and the new
 * relaxation rate.  READING: the collision at time t uses the rate updated from
 * gdot(t), which itself uses omega(t-1).  Optional outputs: rho, u, F, gdot. */
static void collide(const oracle_ctx* o, int64_t k, const double* f, double omega_prev, double* fpost,
                    double* omega_new, double* rho_o, double* u_o, double* F_o, double* gdot_o)
{
    int64_t idx = o->cell[k];
    int x, y, z;
    coords(o, idx, &x, &y, &z);
    double phi = o->phi[idx];
    double rho, u[3], F[3];
    macroscopic(o, f, idx, &rho, u, F);
    double gdot = shear_rate(o, f, phi, rho, u, F, omega_prev);
    double mu = carreau_yasuda(o, gdot);
    double om = omega_of(rho, mu);
    for (int i = 0; i < o->q; ++i) {
        double feq = equilibrium(o, i, phi, rho, u);
        /* Omega^phi_i = w_i rho (phi(x + c_i) - phi(x)) */
        double om_phi = o->w[i] * rho * (link_porosity(o, x, y, z, i, phi) - phi);
        /* Omega^f_i = w_i (1 - omega/2) ((c_i - u)/c_s^2 + (u.c_i) c_i / c_s^4) . rho f */
        double cu = o->c[i][0] * u[0] + o->c[i][1] * u[1] + o->c[i][2] * u[2];
        double gf = 0.0;
        for (int a = 0; a < 3; ++a) gf += ((o->c[i][a] - u[a]) / CS2 + cu * o->c[i][a] / (CS2 * CS2)) * F[a];
        double om_f = o->w[i] * (1.0 - om / 2.0) * gf;
        /* Omega^SRT_i = -omega (f_i - f_i^eq) */
        double om_srt = -om * (f[i] - feq);
        fpost[i] = f[i] + om_phi + om_f + om_srt;
    }
    *omega_new = om;
    if (rho_o) *rho_o = rho;
    if (u_o) for (int a = 0; a < 3; ++a) u_o[a] = u[a];
    if (F_o) for (int a = 0; a < 3; ++a) F_o[a] = F[a];
    if (gdot_o) *gdot_o = gdot;
}

/* ------------------------------------------------------------ boundaries */

/* Mean inflow v(t) = u0 (1 + amp sin(2 pi t / period)), times a linear ramp
 * over the first ramp steps (the pre-run of Sec. 4) when ramp > 0. */
static double inflow_mean(const oracle_ctx* o, int64_t t)
{
    double v = o->p.u0 * (1.0 + o->p.amp * sin(2.0 * M_PI * (double)t / o->p.period));
    if (o->p.ramp > 0.0 && (double)t < o->p.ramp) v *= (double)t / o->p.ramp;
    return v;
}

/* Hagen-Poiseuille inflow (Sec. 4): u_perp(t, r) = 2 v(t) (1 - r^2 / R^2),
 * zero tangential components.  READING: clamped at 0 for centres just outside R. */
static void inlet_velocity(const oracle_ctx* o, int x, int y, int z, int64_t t, double u[3])
{
    double pc[3] = {x + 0.5, y + 0.5, z + 0.5};
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a)
        if (a != o->p.in_axis) r2 += (pc[a] - o->p.in_center[a]) * (pc[a] - o->p.in_center[a]);
    double prof = 1.0 - r2 / (o->p.in_radius * o->p.in_radius);
    if (prof < 0.0) prof = 0.0;
    double un = 2.0 * inflow_mean(o, t) * prof;
    u[0] = u[1] = u[2] = 0.0;
    u[o->p.in_axis] = o->p.in_side == 0 ? un : -un;
}

/* Zou-He velocity inlet (Sec. 4, after Zou & He 1997) in its non-equilibrium
 * bounce-back form for D3Q19/D3Q27.  n is the inward unit normal, U the
 * populations entering from outside (c.n > 0).  With ub = u_in - g/2 (so that
 * the cell's velocity, force shift included, equals u_in; phi = 1 here):
 *   rho = (sum_{c.n=0} f + 2 sum_{c.n<0} f) / (1 - ub.n),
 *   f_i = f_opp(i) + f_i^eq - f_opp(i)^eq            for i in U,
 * which makes sum_i f_i = rho and sum_i f_i c_i.n = rho ub.n exactly; the
 * tangential momentum is rho ub_t + N_t, N_t = sum_{c.n=0} (f - f^eq) c_t.
 * READING: no tangential correction (removing N_t from U, the D2Q9 / D3Q19
 * complement of the scheme).  In D3Q27, spread over the unknowns with c_t != 0
 * or over the edge ones only, that correction makes the inlet linearly
 * unstable at the relaxation times the Carreau-Yasuda law reaches
 * (tau = 0.527 at mu_inf): a perturbed rest state grows by about 5 % per
 * step at the inlet plane, while without it the same state decays. */
static void zou_he_inlet(const oracle_ctx* o, int64_t k, int64_t t)
{
    double* f = o->fnew + k * o->q;
    int64_t idx = o->cell[k];
    int x, y, z;
    coords(o, idx, &x, &y, &z);
    double phi = o->phi[idx];
    int ax = o->p.in_axis;
    int sgn = o->p.in_side == 0 ? 1 : -1;
    double uin[3], ub[3];
    inlet_velocity(o, x, y, z, t, uin);
    for (int a = 0; a < 3; ++a) ub[a] = uin[a] - 0.5 * o->p.g[a];
    double s0 = 0.0, sm = 0.0;
    for (int i = 0; i < o->q; ++i) {
        int cn = o->c[i][ax] * sgn;
        if (cn == 0) s0 += f[i];
        if (cn < 0) sm += f[i];
    }
    double rho = (s0 + 2.0 * sm) / (phi * (1.0 - ub[ax] * sgn));
    for (int i = 0; i < o->q; ++i)
        if (o->c[i][ax] * sgn > 0)
            f[i] = f[o->opp[i]] + equilibrium(o, i, phi, rho, ub) - equilibrium(o, o->opp[i], phi, rho, ub);
}

/* Extrapolation outlet (Sec. 4, after Geier et al. 2015) with prescribed
 * pressure.  READING: non-equilibrium extrapolation from the first interior
 * neighbour nb = x + n (n the inward normal):
 *   f_i(x) = f_i^eq(rho_out, u_nb) + f_i(nb) - f_i^eq(rho_nb, u_nb)   for c_i.n > 0. */
static void extrapolation_outlet(const oracle_ctx* o, int64_t k)
{
    double* f = o->fnew + k * o->q;
    int64_t idx = o->cell[k];
    int x, y, z;
    coords(o, idx, &x, &y, &z);
    int ax = o->p.out_axis;
    int sgn = o->p.out_side == 1 ? -1 : 1;
    int d[3] = {0, 0, 0};
    d[ax] = sgn;
    int fa, fs;
    int64_t nbi = neighbour(o, x, y, z, d, &fa, &fs);
    int64_t kn = o->slot[nbi];
    const double* fn = o->fnew + kn * o->q;
    double rho_nb, u_nb[3], F_nb[3];
    macroscopic(o, fn, nbi, &rho_nb, u_nb, F_nb);
    for (int i = 0; i < o->q; ++i)
        if (o->c[i][ax] * sgn > 0)
            f[i] = equilibrium(o, i, o->phi[idx], o->p.rho_out, u_nb) + fn[i] - equilibrium(o, i, o->phi[nbi], rho_nb, u_nb);
}

static void apply_boundaries(oracle_ctx* o, int64_t t)
{
    int64_t nf = o->nf;
    if (o->p.in_axis >= 0) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k)
            if (o->flags[o->cell[k]] == O_INLET) zou_he_inlet(o, k, t);
    }
    if (o->p.out_axis >= 0) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k)
            if (o->flags[o->cell[k]] == O_OUTLET) extrapolation_outlet(o, k);
    }
}

/* Streaming of the post-collision population of cell k along c_i (push form).
 * Half-way bounce-back (Sec. 4) when the target is solid or the box wall; a
 * population leaving through the inlet/outlet face of an inlet/outlet cell is
 * dropped (it is reconstructed on the other side by the boundary condition). */
static void push_cell(oracle_ctx* o, int64_t k)
{
    int64_t idx = o->cell[k];
    int x, y, z;
    coords(o, idx, &x, &y, &z);
    uint8_t type = o->flags[idx];
    const double* fp = o->fpost + k * o->q;
    for (int i = 0; i < o->q; ++i) {
        int ax, sd;
        int64_t d = neighbour(o, x, y, z, o->c[i], &ax, &sd);
        if (d < 0) {
            int open = (type == O_INLET && ax == o->p.in_axis && sd == o->p.in_side) ||
                       (type == O_OUTLET && ax == o->p.out_axis && sd == o->p.out_side);
            if (!open) o->fnew[k * o->q + o->opp[i]] = fp[i];
        } else if (o->flags[d] == O_SOLID) {
            o->fnew[k * o->q + o->opp[i]] = fp[i];
        } else {
            o->fnew[o->slot[d] * o->q + i] = fp[i];
        }
    }
}

/* ------------------------------------------------------------------ API */

static double lattice_visc(const oracle_params* p, double mu)
{
    /* nu [m^2/s] = mu / rho0, lattice: nu dt / dx^2 (Table 1 scales). */
    return mu / p->rho0 * p->dt / (p->dx * p->dx);
}

/* Error codes: 0 ok, 1 bad argument, 2 out of memory, 3 bad boundary cell. */
oracle_ctx* oracle_create(const oracle_params* p, const uint8_t* flags, const double* phi, int32_t* status)
{
    *status = 1;
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return NULL;
    oracle_ctx* o = (oracle_ctx*)calloc(1, sizeof(oracle_ctx));
    if (!o) { *status = 2; return NULL; }
    o->p = *p;
    if (lattice_build(o)) { free(o); return NULL; }
    o->mu0 = lattice_visc(p, p->mu0);
    o->mu_inf = lattice_visc(p, p->mu_inf);
    o->lam = p->lam / p->dt;
    o->nu_d = p->nu_darcy > 0.0 ? p->nu_darcy * p->dt / (p->dx * p->dx) : o->mu0;
    o->d_p = p->d_p / p->dx;
    o->k_const = p->k_const / (p->dx * p->dx);
    o->n_box = (int64_t)p->nx * p->ny * p->nz;
    o->flags = (uint8_t*)malloc(o->n_box);
    o->phi = (double*)malloc(o->n_box * sizeof(double));
    o->slot = (int64_t*)malloc(o->n_box * sizeof(int64_t));
    if (!o->flags || !o->phi || !o->slot) { *status = 2; return o; }
    memcpy(o->flags, flags, o->n_box);
    memcpy(o->phi, phi, o->n_box * sizeof(double));
    int64_t nf = 0;
    for (int64_t i = 0; i < o->n_box; ++i) o->slot[i] = flags[i] != O_SOLID ? nf++ : -1;
    o->nf = nf;
    o->cell = (int64_t*)malloc((nf ? nf : 1) * sizeof(int64_t));
    size_t fq = (size_t)(nf ? nf : 1) * o->q * sizeof(double);
    o->f = (double*)malloc(fq);
    o->fpost = (double*)malloc(fq);
    o->fnew = (double*)malloc(fq);
    o->omega = (double*)malloc((nf ? nf : 1) * sizeof(double));
    o->omega_new = (double*)malloc((nf ? nf : 1) * sizeof(double));
    if (!o->cell || !o->f || !o->fpost || !o->fnew || !o->omega || !o->omega_new) { *status = 2; return o; }
    for (int64_t i = 0; i < o->n_box; ++i)
        if (o->slot[i] >= 0) o->cell[o->slot[i]] = i;
    /* Boundary cells need phi = 1 (pure fluid) and, for the outlet, a fluid
     * interior neighbour with phi = 1. */
    for (int64_t k = 0; k < nf; ++k) {
        int64_t idx = o->cell[k];
        if (flags[idx] == O_INLET && (p->in_axis < 0 || phi[idx] != 1.0 || p->periodic[p->in_axis])) { *status = 3; return o; }
        if (flags[idx] == O_OUTLET) {
            if (p->out_axis < 0 || phi[idx] != 1.0 || p->periodic[p->out_axis]) { *status = 3; return o; }
            int x, y, z, d[3] = {0, 0, 0}, a, s;
            coords(o, idx, &x, &y, &z);
            d[p->out_axis] = p->out_side == 1 ? -1 : 1;
            int64_t nb = neighbour(o, x, y, z, d, &a, &s);
            if (nb < 0 || flags[nb] != O_FLUID || phi[nb] != 1.0) { *status = 3; return o; }
        }
        if (!(phi[idx] > 0.0)) { *status = 1; return o; }
    }
    /* Initial state: f_i = f_i^eq(rho = 1, u = 0) = w_i phi; omega(-1) = omega(mu0)
     * at rho = 1; then the boundary reconstruction of time 0. */
    for (int64_t k = 0; k < nf; ++k) {
        for (int i = 0; i < o->q; ++i) o->fnew[k * o->q + i] = o->w[i] * o->phi[o->cell[k]];
        o->omega[k] = omega_of(1.0, o->mu0);
    }
    o->t = 0;
    apply_boundaries(o, 0);
    memcpy(o->f, o->fnew, fq);
    *status = 0;
    return o;
}

void oracle_destroy(oracle_ctx* o)
{
    if (!o) return;
    free(o->flags); free(o->phi); free(o->slot); free(o->cell);
    free(o->f); free(o->fpost); free(o->fnew); free(o->omega); free(o->omega_new);
    free(o->aniso_s); free(o->aniso_s_half);
    free(o);
}

/* Anisotropic permeability from now on (see anisotropic_velocity): the shape
 * tensor S and its square root per box cell, [n_box][6] (xx yy zz xy xz yz);
 * NULL returns to the isotropic closure.  Returns 0, or 2 when out of memory. */
int32_t oracle_set_anisotropy(oracle_ctx* o, const double* s, const double* s_half)
{
    free(o->aniso_s); free(o->aniso_s_half);
    o->aniso_s = o->aniso_s_half = NULL;
    if (!s) return 0;
    o->aniso_s = (double*)malloc(o->n_box * 6 * sizeof(double));
    o->aniso_s_half = (double*)malloc(o->n_box * 6 * sizeof(double));
    if (!o->aniso_s || !o->aniso_s_half) {
        free(o->aniso_s); free(o->aniso_s_half);
        o->aniso_s = o->aniso_s_half = NULL;
        return 2;
    }
    memcpy(o->aniso_s, s, o->n_box * 6 * sizeof(double));
    memcpy(o->aniso_s_half, s_half, o->n_box * 6 * sizeof(double));
    return 0;
}

/* n time steps: collide every fluid cell, push, bounce back, reconstruct the
 * inlet and outlet populations of time t+1. */
void oracle_step(oracle_ctx* o, int64_t n)
{
    int64_t nf = o->nf;
    int q = o->q;
    for (int64_t s = 0; s < n; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k)
            collide(o, k, o->f + k * q, o->omega[k], o->fpost + k * q, &o->omega_new[k], 0, 0, 0, 0);
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k) push_cell(o, k);
        apply_boundaries(o, o->t + 1);
        double* tmp = o->f; o->f = o->fnew; o->fnew = tmp;
        tmp = o->omega; o->omega = o->omega_new; o->omega_new = tmp;
        o->t += 1;
    }
}

/* Fields of the current time t on the dense box (0 at solid cells): rho, u,
 * gdot(t) (from omega(t-1)) and omega(t). */
void oracle_moments(const oracle_ctx* o, double* rho, double* ux, double* uy, double* uz, double* gdot,
                    double* omega)
{
    memset(rho, 0, o->n_box * sizeof(double));
    memset(ux, 0, o->n_box * sizeof(double));
    memset(uy, 0, o->n_box * sizeof(double));
    memset(uz, 0, o->n_box * sizeof(double));
    memset(gdot, 0, o->n_box * sizeof(double));
    memset(omega, 0, o->n_box * sizeof(double));
    int64_t nf = o->nf;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        int64_t idx = o->cell[k];
        double phi = o->phi[idx], r, u[3], F[3];
        const double* f = o->f + k * o->q;
        macroscopic(o, f, idx, &r, u, F);
        double g = shear_rate(o, f, phi, r, u, F, o->omega[k]);
        rho[idx] = r; ux[idx] = u[0]; uy[idx] = u[1]; uz[idx] = u[2];
        gdot[idx] = g;
        omega[idx] = omega_of(r, carreau_yasuda(o, g));
    }
}

/* Voxel wall-shear-stress proxy of the current time t (the paper evaluates
 * tau = sigma n - (n . sigma n) n with the outer wall normal n on the wall
 * surface, Sec. 4).  READING (voxel form): at a fluid cell with links to the
 * wall (neighbours that are solid or outside the box, where the step bounces
 * populations back), n = sum over those links of w_i c_i, normalised: the
 * direction of the wall as seen from the cell; sigma = -(1 - omega(t)/2) Pi is
 * the viscous stress recovered from the corrected second moment Pi of
 * shear_rate, with omega(t) the rate of the collision of time t.  Output |tau|
 * in lattice units on the dense box; 0 on cells without wall links, on
 * inlet / outlet cells and on solid cells. */
void oracle_wss(const oracle_ctx* o, double* wss)
{
    memset(wss, 0, o->n_box * sizeof(double));
    int64_t nf = o->nf;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        int64_t idx = o->cell[k];
        if (o->flags[idx] != O_FLUID) continue;
        int x, y, z;
        coords(o, idx, &x, &y, &z);
        double nrm[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < o->q; ++i) {  /* the rest direction adds nothing */
            int ax, sd;
            int64_t d = neighbour(o, x, y, z, o->c[i], &ax, &sd);
            if (d < 0 || o->flags[d] == O_SOLID)
                for (int a = 0; a < 3; ++a) nrm[a] += o->w[i] * o->c[i][a];
        }
        double nn = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        if (!(nn > 1e-12)) continue;
        for (int a = 0; a < 3; ++a) nrm[a] /= nn;
        double phi = o->phi[idx], r, u[3], F[3];
        const double* f = o->f + k * o->q;
        macroscopic(o, f, idx, &r, u, F);
        double pi[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) pi[a][b] = 0.5 * (F[a] * u[b] + u[a] * F[b]);
        for (int i = 0; i < o->q; ++i) {
            double dv = f[i] - equilibrium(o, i, phi, r, u);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) pi[a][b] += dv * o->c[i][a] * o->c[i][b];
        }
        double gd = shear_rate(o, f, phi, r, u, F, o->omega[k]);
        double om = omega_of(r, carreau_yasuda(o, gd));
        double sn[3], nsn = 0.0, t2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            sn[a] = 0.0;
            for (int b = 0; b < 3; ++b) sn[a] += -(1.0 - 0.5 * om) * pi[a][b] * nrm[b];
            nsn += nrm[a] * sn[a];
        }
        for (int a = 0; a < 3; ++a) {
            double ta = sn[a] - nsn * nrm[a];
            t2 += ta * ta;
        }
        wss[idx] = sqrt(t2);
    }
}

/* Diagnostics of the current time: out = {mass sum_x sum_i f_i, kinetic energy
 * sum rho |u|^2 / 2, sum of |u| over the region, region cell count, max |u|,
 * min omega(t), max omega(t), count of non-finite cells}.  region may be NULL
 * (then the region is empty). */
void oracle_diag(const oracle_ctx* o, const uint8_t* region, double* out)
{
    double mass = 0.0, ke = 0.0, rs = 0.0, rc = 0.0, umax = 0.0, omin = 1e300, omax = -1e300, bad = 0.0;
    int64_t nf = o->nf;
#pragma omp parallel for schedule(static) reduction(+ : mass, ke, rs, rc, bad) reduction(max : umax, omax) reduction(min : omin)
    for (int64_t k = 0; k < nf; ++k) {
        int64_t idx = o->cell[k];
        const double* f = o->f + k * o->q;
        double s = 0.0;
        for (int i = 0; i < o->q; ++i) s += f[i];
        double phi = o->phi[idx], r, u[3], F[3];
        macroscopic(o, f, idx, &r, u, F);
        double g = shear_rate(o, f, phi, r, u, F, o->omega[k]);
        double om = omega_of(r, carreau_yasuda(o, g));
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (!isfinite(r) || !isfinite(un) || !isfinite(om)) { bad += 1.0; continue; }
        mass += s;
        ke += 0.5 * r * un * un;
        if (region && region[idx]) { rs += un; rc += 1.0; }
        if (un > umax) umax = un;
        if (om < omin) omin = om;
        if (om > omax) omax = om;
    }
    out[0] = mass; out[1] = ke; out[2] = rs; out[3] = rc; out[4] = umax;
    out[5] = omin; out[6] = omax; out[7] = bad;
}

/* Runs T steps and returns the objective J = (1/T) sum_{t=1..T} (1/|R|)
 * sum_{x in R} rho |u|^2 / 2 over the region R (time-and-region mean kinetic
 * energy of the pre-collision state of each step). */
double oracle_run_objective(oracle_ctx* o, int64_t T, const uint8_t* region)
{
    double acc = 0.0;
    int64_t nf = o->nf;
    for (int64_t s = 0; s < T; ++s) {
        oracle_step(o, 1);
        double ke = 0.0, cnt = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ke, cnt)
        for (int64_t k = 0; k < nf; ++k) {
            int64_t idx = o->cell[k];
            if (!region[idx]) continue;
            double r, u[3], F[3];
            macroscopic(o, o->f + k * o->q, idx, &r, u, F);
            ke += 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            cnt += 1.0;
        }
        acc += cnt > 0.0 ? ke / cnt : 0.0;
    }
    return T > 0 ? acc / (double)T : 0.0;
}

/* ------------------------------------------- introspection for the tests */

int64_t oracle_nfluid(const oracle_ctx* o) { return o->nf; }
int64_t oracle_time(const oracle_ctx* o) { return o->t; }
int32_t oracle_q(const oracle_ctx* o) { return o->q; }

/* Lattice tables in the oracle's own ordering: c [q][3] int32, w [q]. */
void oracle_lattice(const oracle_ctx* o, int32_t* c, double* w, int32_t* opp)
{
    for (int i = 0; i < o->q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = o->c[i][a];
        w[i] = o->w[i];
        opp[i] = o->opp[i];
    }
}

void oracle_cells(const oracle_ctx* o, int64_t* cells) { memcpy(cells, o->cell, o->nf * sizeof(int64_t)); }
void oracle_get_state(const oracle_ctx* o, double* f, double* omega)
{
    memcpy(f, o->f, o->nf * o->q * sizeof(double));
    memcpy(omega, o->omega, o->nf * sizeof(double));
}
void oracle_set_state(oracle_ctx* o, const double* f, const double* omega, int64_t t)
{
    memcpy(o->f, f, o->nf * o->q * sizeof(double));
    memcpy(o->omega, omega, o->nf * sizeof(double));
    o->t = t;
}

/* Collision of fluid cell k on the given populations; out = {rho, ux, uy, uz,
 * Fx, Fy, Fz, gdot, omega_new}. */
void oracle_collide_cell(const oracle_ctx* o, int64_t k, const double* f, double omega_prev, double* fpost,
                         double* out)
{
    double om, r, u[3], F[3], g;
    collide(o, k, f, omega_prev, fpost, &om, &r, u, F, &g);
    out[0] = r; out[1] = u[0]; out[2] = u[1]; out[3] = u[2];
    out[4] = F[0]; out[5] = F[1]; out[6] = F[2]; out[7] = g; out[8] = om;
}

/* Boundary reconstruction alone on the state held in f (time t). */
void oracle_apply_boundaries(oracle_ctx* o, int64_t t)
{
    memcpy(o->fnew, o->f, o->nf * o->q * sizeof(double));
    apply_boundaries(o, t);
    memcpy(o->f, o->fnew, o->nf * o->q * sizeof(double));
}

/* Lattice-unit parameters as the oracle derived them:
 * {mu0, mu_inf, lambda, nu_darcy, d_p, k_const}. */
void oracle_lattice_params(const oracle_ctx* o, double* out)
{
    out[0] = o->mu0; out[1] = o->mu_inf; out[2] = o->lam; out[3] = o->nu_d; out[4] = o->d_p; out[5] = o->k_const;
}

/* Threads the oracle's parallel loops use. */
int32_t oracle_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
