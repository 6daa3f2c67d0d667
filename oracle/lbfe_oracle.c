/*
 * lbfe_oracle.c -- plain FP64 CPU oracle of the hybrid lattice-Boltzmann /
 * finite-difference FENE-P step of Gupta & Sbragaglia, "Deformation and
 * break-up of viscoelastic droplets using Lattice Boltzmann Models".
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA product
 * path never calls it and shares no code, header, table or helper with it.
 *
 * What it computes (Sec. 2 of the paper):
 *   - two immiscible components A (droplet) and B (matrix), each a D3Q19
 *     lattice-Boltzmann population set, coupled by the Shan-Chen
 *     inter-component force (Sec. 2, "Shan-Chen model");
 *   - Navier-Stokes with a composition-weighted viscosity that realises the
 *     total-viscosity ratio lambda of Sec. 2 (Eqs. 1 and 3);
 *   - the FENE-P conformation tensor C advanced by finite differences
 *     (Eqs. 2 and 4) with the Peterlin factor f = (L^2-3)/(L^2-tr C);
 *   - the polymer stress divergence fed back as a body force (last term of
 *     Eqs. 1 and 3);
 *   - walls at z = -1/2 and z = Lz-1/2 moving at -Uw and +Uw along x
 *     (Sec. 3, set-up), periodic x and y.
 * The paper leaves the lattice, the forcing scheme, the FD stencils and the
 * boundary treatment of the FD fields to a companion methodological paper;
 * the readings taken here are, in order:
 *   lattice D3Q19 (w = 1/3, 1/18, 1/36; cs^2 = 1/3);
 *   Shan-Chen force F_s(x) = -G rho_s(x) sum_i w_i rho_t(x+c_i) c_i (t = other
 *     component), densities mirrored across the walls;
 *   Guo forcing with the common barycentric velocity
 *     u = (j_A + j_B + F/2)/rho;
 *   per-site BGK time tau(x) = 3 nu(x) + 1/2, nu = (rho_A nu_A + rho_B nu_B)/rho;
 *   polymer stress Pi = (eta_P/tau_P) chi (f C - I), chi = rho_visc/rho,
 *     F_P = div Pi by central differences;
 *   C^{n+1} = C + [-u.grad C (first-order upwind) + C.grad u + (grad u)^T.C
 *     - (f C - I)/tau_P], (grad u)_ij = d_i u_j by central differences;
 *     optionally (advection = 1) u.grad C by second-order upwind with
 *     minmod-limited slopes;
 *   FD ghosts at the walls: C and rho mirrored, u_ghost = 2 U_wall - u;
 *   halfway bounce-back with the moving-wall momentum term.
 * One step performs, over full fields and in this order: moments, Shan-Chen
 * force, polymer stress and its divergence, velocity, FENE-P update,
 * collision, streaming.  The LB force uses C^n; C^{n+1} uses u^n.
 *
 * Pins (tests/test_oracle_*.py): Couette and Poiseuille solutions, exact
 * mass conservation, the Guo moment identities, closed forms of the
 * Shan-Chen and polymer forces, flat-interface coexistence and the Laplace
 * law, Eqs. 6 and 7 in steady shear, the Oldroyd-B start-up, the stencils'
 * exact properties (including the second-order advection on quadratics and
 * its boundedness), and the observables on built shapes.  The coupled
 * droplet dynamics as a whole have no closed form: parity unpinned beyond
 * these pins.
 *
 * Layout (shared interface format, restated independently on the GPU side):
 *   cell index n = (z*Ly + y)*Lx + x;
 *   f[(s*19 + i)*N + n], s = 0 (A) / 1 (B), i in the velocity order below;
 *   C[k*N + n], k = xx, yy, zz, xy, xz, yz.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities: rest, 6 faces, 12 edges; opposite of i>0 is i^1 paired
 * as (1,2),(3,4),... */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static double weight(int i) {
    int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i) {
    for (int k = 0; k < Q; ++k)
        if (CX[k] == -CX[i] && CY[k] == -CY[i] && CZ[k] == -CZ[i]) return k;
    return -1;
}

typedef struct {
    int Lx, Ly, Lz;       /* lattice; the wall gap W equals Lz */
    int visco_phase;      /* 0 Newtonian, 1 viscoelastic droplet (DV), 2 viscoelastic matrix (MV) */
    double Uw;            /* wall speed: bottom wall -Uw, top wall +Uw, along x */
    double G;             /* Shan-Chen inter-component coupling */
    double eta_M;         /* matrix total dynamic viscosity */
    double lambda;        /* droplet/matrix total-viscosity ratio */
    double eta_P;         /* polymer viscosity of the viscoelastic phase */
    double tau_P;         /* polymer relaxation time */
    double L2;            /* FENE-P extensibility L^2 */
    double rho_in;        /* bulk density of a component where it is the majority */
    double rho_out;       /* bulk density of the dissolved (minority) component */
    double gx, gy, gz;    /* constant body acceleration (verification hook) */
    int advection;        /* u.grad C: 0 first-order upwind, 1 second-order minmod-limited upwind */
} orc_params;

typedef struct {
    double nu_A, nu_B;    /* kinematic viscosities of the two Newtonian solvents */
    double pi_coef;       /* eta_P / tau_P of the viscoelastic phase (0 if Newtonian) */
    int visc_comp;        /* component carrying the polymer: 0 (A), 1 (B), -1 none */
} orc_derived;

/* Sec. 2: lambda = eta_d/eta_M with total (solvent + polymer) viscosities.
 * DV: eta_d = eta_A + eta_P, eta_M = eta_B.  MV: eta_d = eta_A,
 * eta_M = eta_B + eta'_P.  Kinematic viscosities use the bulk total density
 * rho_in + rho_out, which is the same in both phases. */
int orc_derive(const orc_params *p, orc_derived *d) {
    double rho_ref = p->rho_in + p->rho_out;
    double eta_d = p->lambda * p->eta_M;
    double eta_A = eta_d, eta_B = p->eta_M;
    d->pi_coef = 0.0;
    d->visc_comp = -1;
    if (p->visco_phase == 1) {
        eta_A = eta_d - p->eta_P;
        d->pi_coef = p->eta_P / p->tau_P;
        d->visc_comp = 0;
    } else if (p->visco_phase == 2) {
        eta_B = p->eta_M - p->eta_P;
        d->pi_coef = p->eta_P / p->tau_P;
        d->visc_comp = 1;
    }
    d->nu_A = eta_A / rho_ref;
    d->nu_B = eta_B / rho_ref;
    if (!(d->nu_A > 0.0) || !(d->nu_B > 0.0) || !(p->tau_P > 0.0) || !(p->L2 > 3.0)) return 1;
    return 0;
}

static size_t ncell(const orc_params *p) { return (size_t)p->Lx * p->Ly * p->Lz; }

static size_t idx(const orc_params *p, int x, int y, int z) {
    return ((size_t)z * p->Ly + y) * p->Lx + x;
}

static int wrap(int a, int L) { return ((a % L) + L) % L; }
static int clampz(int z, int Lz) { return z < 0 ? 0 : (z >= Lz ? Lz - 1 : z); }

/* f^eq_i(rho, u) = w_i rho [1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)] */
static double feq(int i, double rho, double ux, double uy, double uz) {
    double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
    double uu = ux * ux + uy * uy + uz * uz;
    return weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Initial state: f = f^eq(rho_s, u = 0), C = I. */
void orc_init(const orc_params *p, const double *rho_init, double *f, double *C) {
    size_t N = ncell(p);
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < Q; ++i)
            for (size_t n = 0; n < N; ++n)
                f[((size_t)s * Q + i) * N + n] = feq(i, rho_init[(size_t)s * N + n], 0.0, 0.0, 0.0);
    for (size_t n = 0; n < N; ++n) {
        C[0 * N + n] = 1.0; C[1 * N + n] = 1.0; C[2 * N + n] = 1.0;
        C[3 * N + n] = 0.0; C[4 * N + n] = 0.0; C[5 * N + n] = 0.0;
    }
}

/* Component densities and momenta of the streamed state. */
void orc_moments(const orc_params *p, const double *f, double *rho /*[2][N]*/, double *jm /*[2][3][N]*/) {
    size_t N = ncell(p);
    #pragma omp parallel for schedule(static)
    for (long long nn = 0; nn < (long long)N; ++nn) {
        size_t n = (size_t)nn;
        for (int s = 0; s < 2; ++s) {
            double r = 0, jx = 0, jy = 0, jz = 0;
            for (int i = 0; i < Q; ++i) {
                double v = f[((size_t)s * Q + i) * N + n];
                r += v; jx += v * CX[i]; jy += v * CY[i]; jz += v * CZ[i];
            }
            rho[(size_t)s * N + n] = r;
            jm[((size_t)s * 3 + 0) * N + n] = jx;
            jm[((size_t)s * 3 + 1) * N + n] = jy;
            jm[((size_t)s * 3 + 2) * N + n] = jz;
        }
    }
}

/* Shan-Chen inter-component force, psi = rho:
 * F_s(x) = -G rho_s(x) sum_i w_i rho_t(x + c_i) c_i, t = other component.
 * Neighbours beyond a wall read the adjacent fluid layer (mirror). */
void orc_sc_force(const orc_params *p, const double *rho, double *Fsc /*[2][3][N]*/) {
    size_t N = ncell(p);
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < p->Lz; ++z)
        for (int y = 0; y < p->Ly; ++y)
            for (int x = 0; x < p->Lx; ++x) {
                size_t n = idx(p, x, y, z);
                for (int s = 0; s < 2; ++s) {
                    const double *other = rho + (size_t)(1 - s) * N;
                    double sx = 0, sy = 0, sz = 0;
                    for (int i = 1; i < Q; ++i) {
                        size_t m = idx(p, wrap(x + CX[i], p->Lx), wrap(y + CY[i], p->Ly), clampz(z + CZ[i], p->Lz));
                        double wr = weight(i) * other[m];
                        sx += wr * CX[i]; sy += wr * CY[i]; sz += wr * CZ[i];
                    }
                    double pre = -p->G * rho[(size_t)s * N + n];
                    Fsc[((size_t)s * 3 + 0) * N + n] = pre * sx;
                    Fsc[((size_t)s * 3 + 1) * N + n] = pre * sy;
                    Fsc[((size_t)s * 3 + 2) * N + n] = pre * sz;
                }
            }
}

/* Peterlin factor of Eq. 2: f(r_P) = (L^2 - 3)/(L^2 - r_P^2), r_P^2 = tr C. */
static double peterlin(double L2, double trC) { return (L2 - 3.0) / (L2 - trC); }

/* Polymer stress Pi = (eta_P/tau_P) chi (f C - I), chi = rho_visc/rho
 * (last term of Eqs. 1 and 3, written in the form that exerts no force where
 * the polymer fraction is uniform and C = I). */
void orc_polymer_stress(const orc_params *p, const orc_derived *d, const double *rho, const double *C, double *Pi /*[6][N]*/) {
    size_t N = ncell(p);
    for (size_t n = 0; n < N; ++n) {
        double chi = 0.0;
        if (d->visc_comp >= 0) chi = rho[(size_t)d->visc_comp * N + n] / (rho[n] + rho[N + n]);
        double trC = C[0 * N + n] + C[1 * N + n] + C[2 * N + n];
        double fp = peterlin(p->L2, trC);
        double a = d->pi_coef * chi;
        for (int k = 0; k < 6; ++k) {
            double delta = k < 3 ? 1.0 : 0.0;
            Pi[(size_t)k * N + n] = a * (fp * C[(size_t)k * N + n] - delta);
        }
    }
}

/* symmetric-tensor component index for (a,b), a,b in {0,1,2} */
static int sym(int a, int b) {
    static const int T[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    return T[a][b];
}

/* F_P,a(x) = sum_b d_b Pi_ba, second-order central differences; Pi beyond a
 * wall equals Pi of the adjacent layer (C and rho both mirrored). */
void orc_polymer_force(const orc_params *p, const double *Pi, double *FP /*[3][N]*/) {
    size_t N = ncell(p);
    for (int z = 0; z < p->Lz; ++z)
        for (int y = 0; y < p->Ly; ++y)
            for (int x = 0; x < p->Lx; ++x) {
                size_t n = idx(p, x, y, z);
                size_t nb[3][2] = {
                    {idx(p, wrap(x + 1, p->Lx), y, z), idx(p, wrap(x - 1, p->Lx), y, z)},
                    {idx(p, x, wrap(y + 1, p->Ly), z), idx(p, x, wrap(y - 1, p->Ly), z)},
                    {idx(p, x, y, clampz(z + 1, p->Lz)), idx(p, x, y, clampz(z - 1, p->Lz))}};
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < 3; ++b) {
                        int k = sym(b, a);
                        s += 0.5 * (Pi[(size_t)k * N + nb[b][0]] - Pi[(size_t)k * N + nb[b][1]]);
                    }
                    FP[(size_t)a * N + n] = s;
                }
            }
}

/* Velocity with the Guo half-force shift and the per-component total forces
 * F_s,tot = F_s^SC + (rho_s/rho) F_P + rho_s g. */
void orc_velocity(const orc_params *p, const double *rho, const double *jm, const double *Fsc,
                  const double *FP, double *u /*[3][N]*/, double *Ftot /*[2][3][N]*/) {
    size_t N = ncell(p);
    double g[3] = {p->gx, p->gy, p->gz};
    for (size_t n = 0; n < N; ++n) {
        double rt = rho[n] + rho[N + n];
        for (int a = 0; a < 3; ++a) {
            double Fsum = 0.0, jsum = 0.0;
            for (int s = 0; s < 2; ++s) {
                double rs = rho[(size_t)s * N + n];
                double Fs = Fsc[((size_t)s * 3 + a) * N + n] + (rs / rt) * FP[(size_t)a * N + n] + rs * g[a];
                Ftot[((size_t)s * 3 + a) * N + n] = Fs;
                Fsum += Fs;
                jsum += jm[((size_t)s * 3 + a) * N + n];
            }
            u[(size_t)a * N + n] = (jsum + 0.5 * Fsum) / rt;
        }
    }
}

/* Velocity at (x, y, z) with the wall ghost rule u_ghost = 2 U_wall - u. */
static double u_at(const orc_params *p, const double *u, int a, int x, int y, int z) {
    size_t N = ncell(p);
    x = wrap(x, p->Lx); y = wrap(y, p->Ly);
    if (z < 0) {
        double uw = (a == 0) ? -p->Uw : 0.0;
        return 2.0 * uw - u[(size_t)a * N + idx(p, x, y, 0)];
    }
    if (z >= p->Lz) {
        double uw = (a == 0) ? p->Uw : 0.0;
        return 2.0 * uw - u[(size_t)a * N + idx(p, x, y, p->Lz - 1)];
    }
    return u[(size_t)a * N + idx(p, x, y, z)];
}

static double C_at(const orc_params *p, const double *C, int k, int x, int y, int z) {
    size_t N = ncell(p);
    return C[(size_t)k * N + idx(p, wrap(x, p->Lx), wrap(y, p->Ly), clampz(z, p->Lz))];
}

/* minmod limiter: 0 where the two differences disagree in sign, else the
 * one of smaller magnitude. */
static double minmod(double a, double b) {
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* Second-order upwind derivative of component k along the unit vector e at
 * (x, y, z) for a velocity component v (a reading: the paper defers its FD
 * scheme).  With the limited slope s_j = minmod(C_{j+1} - C_j, C_j - C_{j-1})
 * and face values reconstructed from the upwind side,
 *   v > 0:  D = (C_0 + s_0/2) - (C_-1 + s_-1/2),
 *   v <= 0: D = (C_1 - s_1/2) - (C_0 - s_0/2).
 * Offsets past a wall take the wall cell's value (zero gradient, as for the
 * first-order scheme); x and y are periodic. */
static double d_upwind2(const orc_params *p, const double *C, int k, int x, int y, int z, const int e[3], double v) {
    double c[5];
    for (int j = -2; j <= 2; ++j) c[j + 2] = C_at(p, C, k, x + j * e[0], y + j * e[1], z + j * e[2]);
    const double sm = minmod(c[2] - c[1], c[1] - c[0]);   /* slope at offset -1 */
    const double s0 = minmod(c[3] - c[2], c[2] - c[1]);   /* slope at offset 0 */
    const double sp = minmod(c[4] - c[3], c[3] - c[2]);   /* slope at offset +1 */
    if (v > 0.0) return (c[2] + 0.5 * s0) - (c[1] + 0.5 * sm);
    return (c[3] - 0.5 * sp) - (c[2] - 0.5 * s0);
}

/* FENE-P finite-difference update, Eq. 2 (and Eq. 4 for the matrix):
 * C^{n+1} = C + [ -u.grad C + C.(grad u) + (grad u)^T.C - (f C - I)/tau_P ]
 * with (grad u)_ij = d_i u_j (central), u.grad C upwind (first order, or
 * second order with the minmod limiter when advection = 1), dt = 1. */
void orc_fene_update(const orc_params *p, const double *C, const double *u, double *Cn) {
    size_t N = ncell(p);
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < p->Lz; ++z)
        for (int y = 0; y < p->Ly; ++y)
            for (int x = 0; x < p->Lx; ++x) {
                size_t n = idx(p, x, y, z);
                int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                double Gr[3][3]; /* Gr[i][j] = d_i u_j */
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        Gr[i][j] = 0.5 * (u_at(p, u, j, x + e[i][0], y + e[i][1], z + e[i][2]) -
                                          u_at(p, u, j, x - e[i][0], y - e[i][1], z - e[i][2]));
                double uc[3] = {u[n], u[N + n], u[2 * N + n]};
                double Cm[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Cm[i][j] = C[(size_t)sym(i, j) * N + n];
                double trC = Cm[0][0] + Cm[1][1] + Cm[2][2];
                double fp = peterlin(p->L2, trC);
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 3; ++j) {
                        int k = sym(i, j);
                        double adv = 0.0;
                        for (int b = 0; b < 3; ++b) {
                            double c0 = Cm[i][j];
                            if (p->advection == 1) {
                                adv += uc[b] * d_upwind2(p, C, k, x, y, z, e[b], uc[b]);
                            } else if (uc[b] > 0.0) {
                                double cm = C_at(p, C, k, x - e[b][0], y - e[b][1], z - e[b][2]);
                                adv += uc[b] * (c0 - cm);
                            } else {
                                double cp = C_at(p, C, k, x + e[b][0], y + e[b][1], z + e[b][2]);
                                adv += uc[b] * (cp - c0);
                            }
                        }
                        double stretch = 0.0;
                        for (int m = 0; m < 3; ++m) stretch += Cm[i][m] * Gr[m][j] + Gr[m][i] * Cm[m][j];
                        double relax = (fp * Cm[i][j] - (i == j ? 1.0 : 0.0)) / p->tau_P;
                        Cn[(size_t)k * N + n] = Cm[i][j] + (-adv + stretch - relax);
                    }
            }
}

/* BGK collision with per-site tau and the Guo source term, per component:
 * f*_i = f_i - (f_i - f^eq_i(rho_s, u))/tau
 *        + (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F_s,tot */
void orc_collide(const orc_params *p, const orc_derived *d, const double *f, const double *rho,
                 const double *u, const double *Ftot, double *fpost) {
    size_t N = ncell(p);
    #pragma omp parallel for schedule(static)
    for (long long nn = 0; nn < (long long)N; ++nn) {
        size_t n = (size_t)nn;
        double rA = rho[n], rB = rho[N + n], rt = rA + rB;
        double nu = (rA * d->nu_A + rB * d->nu_B) / rt;
        double tau = 3.0 * nu + 0.5;
        double ux = u[n], uy = u[N + n], uz = u[2 * N + n];
        for (int s = 0; s < 2; ++s) {
            double rs = rho[(size_t)s * N + n];
            double Fx = Ftot[((size_t)s * 3 + 0) * N + n];
            double Fy = Ftot[((size_t)s * 3 + 1) * N + n];
            double Fz = Ftot[((size_t)s * 3 + 2) * N + n];
            for (int i = 0; i < Q; ++i) {
                size_t a = ((size_t)s * Q + i) * N + n;
                double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
                double src = (1.0 - 0.5 / tau) * weight(i) *
                             ((3.0 * (CX[i] - ux) + 9.0 * cu * CX[i]) * Fx +
                              (3.0 * (CY[i] - uy) + 9.0 * cu * CY[i]) * Fy +
                              (3.0 * (CZ[i] - uz) + 9.0 * cu * CZ[i]) * Fz);
                fpost[a] = f[a] - (f[a] - feq(i, rs, ux, uy, uz)) / tau + src;
            }
        }
    }
}

/* Pull streaming with halfway bounce-back at z = -1/2 (wall velocity -Uw)
 * and z = Lz - 1/2 (+Uw): a population whose source x - c_i lies in a wall is
 * the reflected post-collision population of the same cell plus the
 * moving-wall term 2 w_i rho_s (c_i . U_wall)/cs^2. */
void orc_stream(const orc_params *p, const double *fpost, const double *rho, double *fnew) {
    size_t N = ncell(p);
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < p->Lz; ++z)
        for (int y = 0; y < p->Ly; ++y)
            for (int x = 0; x < p->Lx; ++x) {
                size_t n = idx(p, x, y, z);
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < Q; ++i) {
                        int zs = z - CZ[i];
                        double v;
                        if (zs < 0 || zs >= p->Lz) {
                            double uw = zs < 0 ? -p->Uw : p->Uw;
                            v = fpost[((size_t)s * Q + opposite(i)) * N + n] +
                                2.0 * weight(i) * rho[(size_t)s * N + n] * (CX[i] * uw) * 3.0;
                        } else {
                            size_t m = idx(p, wrap(x - CX[i], p->Lx), wrap(y - CY[i], p->Ly), zs);
                            v = fpost[((size_t)s * Q + i) * N + m];
                        }
                        fnew[((size_t)s * Q + i) * N + n] = v;
                    }
            }
}

/* Everything of one step up to the collision, exposing the intermediate
 * fields (any output pointer may be NULL).  f and C are not modified. */
int orc_step_detail(const orc_params *p, const double *f, const double *C, double *fpost_out,
                    double *rho_out, double *u_out, double *Ftot_out, double *Cnew_out) {
    orc_derived d;
    if (orc_derive(p, &d)) return 1;
    size_t N = ncell(p);
    double *rho = malloc(sizeof(double) * 2 * N);
    double *jm = malloc(sizeof(double) * 6 * N);
    double *Fsc = malloc(sizeof(double) * 6 * N);
    double *Pi = malloc(sizeof(double) * 6 * N);
    double *FP = malloc(sizeof(double) * 3 * N);
    double *u = malloc(sizeof(double) * 3 * N);
    double *Ftot = malloc(sizeof(double) * 6 * N);
    double *Cn = malloc(sizeof(double) * 6 * N);
    double *fpost = malloc(sizeof(double) * 2 * Q * N);
    if (!rho || !jm || !Fsc || !Pi || !FP || !u || !Ftot || !Cn || !fpost) {
        free(rho); free(jm); free(Fsc); free(Pi); free(FP); free(u); free(Ftot); free(Cn); free(fpost);
        return 2;
    }
    orc_moments(p, f, rho, jm);                           /* 1 */
    orc_sc_force(p, rho, Fsc);                            /* 2 */
    orc_polymer_stress(p, &d, rho, C, Pi);                /* 3 */
    orc_polymer_force(p, Pi, FP);
    orc_velocity(p, rho, jm, Fsc, FP, u, Ftot);           /* 4 */
    orc_fene_update(p, C, u, Cn);                         /* 5 */
    orc_collide(p, &d, f, rho, u, Ftot, fpost);           /* 6 */
    if (fpost_out) memcpy(fpost_out, fpost, sizeof(double) * 2 * Q * N);
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * 2 * N);
    if (u_out) memcpy(u_out, u, sizeof(double) * 3 * N);
    if (Ftot_out) memcpy(Ftot_out, Ftot, sizeof(double) * 6 * N);
    if (Cnew_out) memcpy(Cnew_out, Cn, sizeof(double) * 6 * N);
    free(rho); free(jm); free(Fsc); free(Pi); free(FP); free(u); free(Ftot); free(Cn); free(fpost);
    return 0;
}

/* n full steps in place on (f, C). */
int orc_step(const orc_params *p, double *f, double *C, long long nsteps) {
    size_t N = ncell(p);
    double *fpost = malloc(sizeof(double) * 2 * Q * N);
    double *rho = malloc(sizeof(double) * 2 * N);
    double *Cn = malloc(sizeof(double) * 6 * N);
    if (!fpost || !rho || !Cn) { free(fpost); free(rho); free(Cn); return 2; }
    int rc = 0;
    for (long long t = 0; t < nsteps && rc == 0; ++t) {
        rc = orc_step_detail(p, f, C, fpost, rho, NULL, NULL, Cn);
        if (rc) break;
        orc_stream(p, fpost, rho, f);                     /* 7 */
        memcpy(C, Cn, sizeof(double) * 6 * N);
    }
    free(fpost); free(rho); free(Cn);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Droplet observables.  The paper measures deformation and orientation
 * (Sec. 1, Sec. 3), the projected length L_p on the flow direction (Sec. 3,
 * Fig. 3) and break-up with multiple necking (Sec. 3, Figs. 2 and 4) without
 * printing their formulas; the readings are:
 *   droplet set S = {cells with rho_A > rho_B};
 *   A(x) = number of droplet cells in the plane x (periodic in x);
 *   L_p = Lx minus the longest circular run of empty planes; the unwrapped
 *     coordinate x' is measured from the first occupied plane after that run;
 *   D = (a - b)/(a + b), a, b = sqrt(5 mu/V) for the largest/smallest
 *     eigenvalues mu of the second-moment tensor of S (uniform ellipsoid);
 *   theta = angle of the major axis in the x-z plane from +x, in (-90, 90];
 *   a neck is an interior local minimum of A that is not empty (an empty
 *     plane separates fragments) and lies below half the smaller of the two
 *     adjacent maxima (plateaus taken at their first plane);
 *   break-up: at least two separated occupied runs of A each holding at
 *     least 1% of the droplet volume.
 * With indicator_fp32 set, rho_A and rho_B are summed in single precision in
 * the population order, which is how the single-precision GPU path decides
 * membership; both then take the same integer decisions.
 * ------------------------------------------------------------------------- */
typedef struct {
    double mass[2];
    double volume;
    double centroid[3];
    double D, theta_deg, Lp;
    double M[6];          /* second moments xx, yy, zz, xy, xz, yz about the centroid */
    int necks, fragments, broken, nan_seen;
} orc_obs;

/* Jacobi eigen-decomposition of a symmetric 3x3 matrix (classical cyclic
 * rotations); eigenvalues in ev, eigenvectors in the columns of V. */
static void jacobi3(double A[3][3], double ev[3], double V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (off < 1e-300) break;
        for (int pq = 0; pq < 3; ++pq) {
            int P = pq == 2 ? 1 : 0, R = pq == 0 ? 1 : 2;
            if (A[P][R] == 0.0) continue;
            double th = (A[R][R] - A[P][P]) / (2.0 * A[P][R]);
            double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            for (int k = 0; k < 3; ++k) { /* A <- A J */
                double akp = A[k][P], akr = A[k][R];
                A[k][P] = c * akp - s * akr;
                A[k][R] = s * akp + c * akr;
            }
            for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                double apk = A[P][k], ark = A[R][k];
                A[P][k] = c * apk - s * ark;
                A[R][k] = s * apk + c * ark;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = V[k][P], vkr = V[k][R];
                V[k][P] = c * vkp - s * vkr;
                V[k][R] = s * vkp + c * vkr;
            }
        }
    }
    for (int i = 0; i < 3; ++i) ev[i] = A[i][i];
}

void orc_eig3(const double *Msym /*xx,yy,zz,xy,xz,yz*/, double *ev, double *V /*3x3 row-major, columns = vectors*/) {
    double A[3][3] = {{Msym[0], Msym[3], Msym[4]}, {Msym[3], Msym[1], Msym[5]}, {Msym[4], Msym[5], Msym[2]}};
    double VV[3][3];
    jacobi3(A, ev, VV);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i * 3 + j] = VV[i][j];
}

/* Profile analysis shared by the field observables and the unit tests:
 * from A(x) (length Lx) compute L_p, the start plane of the unwrapped axis,
 * the neck count and the number of fragments holding >= 1% of the volume. */
void orc_profile(const long long *A, int Lx, int *Lp_out, int *start_out, int *necks_out, int *frag_out) {
    long long V = 0;
    for (int x = 0; x < Lx; ++x) V += A[x];
    if (V == 0) { *Lp_out = 0; *start_out = 0; *necks_out = 0; *frag_out = 0; return; }
    /* longest circular run of empty planes */
    int best_len = 0, best_end = -1;
    for (int x0 = 0; x0 < Lx; ++x0) {
        if (A[x0] != 0) continue;
        if (A[wrap(x0 - 1, Lx)] == 0) continue; /* not the start of a run */
        int len = 0;
        while (len < Lx && A[wrap(x0 + len, Lx)] == 0) ++len;
        if (len > best_len) { best_len = len; best_end = x0 + len; }
    }
    int start = best_len > 0 ? wrap(best_end, Lx) : 0;
    int Lp = Lx - best_len;
    /* sequence along the unwrapped axis */
    long long *a = malloc(sizeof(long long) * (size_t)Lp);
    for (int k = 0; k < Lp; ++k) a[k] = A[wrap(start + k, Lx)];
    /* fragments: maximal runs of occupied planes */
    int frag = 0;
    for (int k = 0; k < Lp;) {
        if (a[k] == 0) { ++k; continue; }
        long long vol = 0;
        while (k < Lp && a[k] != 0) vol += a[k++];
        if (100 * vol >= V) ++frag;
    }
    /* necks: alternate extrema of the plateau-compressed sequence, framed by
     * empty planes at both ends */
    int m = 0;
    long long *c = malloc(sizeof(long long) * (size_t)(Lp + 2));
    c[m++] = 0;
    for (int k = 0; k < Lp; ++k)
        if (a[k] != c[m - 1]) c[m++] = a[k];
    if (c[m - 1] != 0) c[m++] = 0;
    int necks = 0;
    long long last_max = -1;
    int have_min = 0;
    long long pend_min = 0;
    for (int k = 1; k + 1 < m; ++k) {
        if (c[k] > c[k - 1] && c[k] > c[k + 1]) { /* local maximum */
            if (have_min && last_max >= 0) {
                long long lo = last_max < c[k] ? last_max : c[k];
                if (pend_min > 0 && 2 * pend_min < lo) ++necks;
            }
            last_max = c[k];
            have_min = 0;
        } else if (c[k] < c[k - 1] && c[k] < c[k + 1]) { /* local minimum */
            pend_min = c[k];
            have_min = 1;
        }
    }
    free(a); free(c);
    *Lp_out = Lp; *start_out = start; *necks_out = necks; *frag_out = frag;
}

int orc_observables(const orc_params *p, const double *f, int indicator_fp32, orc_obs *o) {
    size_t N = ncell(p);
    int Lx = p->Lx, Ly = p->Ly, Lz = p->Lz;
    long long *A = calloc((size_t)Lx, sizeof(long long));
    /* per-plane integer sums: count, sum y, sum z, sum y^2, sum z^2, sum yz */
    long long *Sy = calloc((size_t)Lx, sizeof(long long)), *Sz = calloc((size_t)Lx, sizeof(long long));
    long long *Syy = calloc((size_t)Lx, sizeof(long long)), *Szz = calloc((size_t)Lx, sizeof(long long));
    long long *Syz = calloc((size_t)Lx, sizeof(long long));
    memset(o, 0, sizeof(*o));
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                size_t n = idx(p, x, y, z);
                double r[2];
                for (int s = 0; s < 2; ++s) {
                    double acc = 0.0;
                    for (int i = 0; i < Q; ++i) acc += f[((size_t)s * Q + i) * N + n];
                    r[s] = acc;
                    o->mass[s] += acc;
                }
                int in;
                if (indicator_fp32) {
                    float ra = 0.0f, rb = 0.0f;
                    for (int i = 0; i < Q; ++i) {
                        ra += (float)f[((size_t)0 * Q + i) * N + n];
                        rb += (float)f[((size_t)1 * Q + i) * N + n];
                    }
                    in = ra > rb;
                    if (ra != ra || rb != rb) o->nan_seen = 1;
                } else {
                    in = r[0] > r[1];
                    if (r[0] != r[0] || r[1] != r[1]) o->nan_seen = 1;
                }
                if (in) {
                    A[x] += 1; Sy[x] += y; Sz[x] += z;
                    Syy[x] += (long long)y * y; Szz[x] += (long long)z * z; Syz[x] += (long long)y * z;
                }
            }
    int Lp, start, necks, frag;
    orc_profile(A, Lx, &Lp, &start, &necks, &frag);
    o->Lp = Lp; o->necks = necks; o->fragments = frag; o->broken = frag >= 2;
    /* moments with x' = (x - start) mod Lx */
    double V = 0, sx = 0, sy = 0, sz = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int x = 0; x < Lx; ++x) {
        double xp = (double)wrap(x - start, Lx);
        V += (double)A[x];
        sx += xp * (double)A[x]; sxx += xp * xp * (double)A[x];
        sy += (double)Sy[x]; sz += (double)Sz[x];
        syy += (double)Syy[x]; szz += (double)Szz[x]; syz += (double)Syz[x];
        sxy += xp * (double)Sy[x]; sxz += xp * (double)Sz[x];
    }
    o->volume = V;
    if (V > 0) {
        double cx = sx / V, cy = sy / V, cz = sz / V;
        o->centroid[0] = fmod(cx + start, (double)Lx);
        o->centroid[1] = cy; o->centroid[2] = cz;
        o->M[0] = sxx - V * cx * cx; o->M[1] = syy - V * cy * cy; o->M[2] = szz - V * cz * cz;
        o->M[3] = sxy - V * cx * cy; o->M[4] = sxz - V * cx * cz; o->M[5] = syz - V * cy * cz;
        double ev[3], Vec[9];
        orc_eig3(o->M, ev, Vec);
        int imax = 0, imin = 0;
        for (int k = 1; k < 3; ++k) {
            if (ev[k] > ev[imax]) imax = k;
            if (ev[k] < ev[imin]) imin = k;
        }
        double a = sqrt(5.0 * fmax(ev[imax], 0.0) / V), b = sqrt(5.0 * fmax(ev[imin], 0.0) / V);
        o->D = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
        double vx = Vec[0 * 3 + imax], vz = Vec[2 * 3 + imax];
        double th = atan2(vz, vx) * 180.0 / M_PI;
        if (th <= -90.0) th += 180.0;
        if (th > 90.0) th -= 180.0;
        o->theta_deg = th;
    }
    free(A); free(Sy); free(Sz); free(Syy); free(Szz); free(Syz);
    return 0;
}

/* 6-connected component count of the droplet set (periodic x and y), with
 * components below 1% of the droplet volume ignored.  Cross-check of the
 * profile-based break-up flag. */
int orc_count_components(const orc_params *p, const double *f) {
    size_t N = ncell(p);
    int *lab = malloc(sizeof(int) * N);
    int *stack = malloc(sizeof(int) * N);
    unsigned char *in = malloc(N);
    long long V = 0;
    for (size_t n = 0; n < N; ++n) {
        double r0 = 0, r1 = 0;
        for (int i = 0; i < Q; ++i) { r0 += f[(size_t)i * N + n]; r1 += f[((size_t)Q + i) * N + n]; }
        in[n] = r0 > r1;
        V += in[n];
        lab[n] = -1;
    }
    int count = 0;
    for (size_t n0 = 0; n0 < N; ++n0) {
        if (!in[n0] || lab[n0] >= 0) continue;
        long long vol = 0;
        int sp = 0;
        stack[sp++] = (int)n0;
        lab[n0] = 1;
        while (sp) {
            int n = stack[--sp];
            ++vol;
            int x = n % p->Lx, y = (n / p->Lx) % p->Ly, z = n / (p->Lx * p->Ly);
            int nb[6][3] = {{x + 1, y, z}, {x - 1, y, z}, {x, y + 1, z}, {x, y - 1, z}, {x, y, z + 1}, {x, y, z - 1}};
            for (int k = 0; k < 6; ++k) {
                int zz = nb[k][2];
                if (zz < 0 || zz >= p->Lz) continue;
                size_t m = idx(p, wrap(nb[k][0], p->Lx), wrap(nb[k][1], p->Ly), zz);
                if (in[m] && lab[m] < 0) { lab[m] = 1; stack[sp++] = (int)m; }
            }
        }
        if (100 * vol >= V) ++count;
    }
    free(lab); free(stack); free(in);
    return count;
}

/* Size of the parameter struct, so that the caller can check its marshalling. */
size_t orc_params_size(void) { return sizeof(orc_params); }
size_t orc_obs_size(void) { return sizeof(orc_obs); }
