/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the reactive two-component
 * lattice Boltzmann capillary-infiltration step (Sergi, Grossi, Leidi,
 * Ortona, arXiv:1309.6726).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a checker library
 * that tests, the smoke check and the benchmark's CPU-baseline leg call.
 * No product code path links, loads or calls it, and it shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes (paper Sec. II, "LB models"):
 *   - two-component D2Q9 BGK, one population set per component
 *     (A = wetting melt, B = the displaced substance);
 *   - bounce-back at the fluid-solid interface (half-way / link form);
 *   - Martys-Chen cohesive (fluid-fluid) and adhesive (fluid-solid) forces,
 *     applied with the Shan-Chen shift of the equilibrium velocity;
 *   - a solute (reactant) concentration C carried by a D2Q4 BGK
 *     advection-diffusion lattice, weakly coupled to the fluid velocity;
 *   - a first-order surface reaction with rate constant k_r at fluid nodes
 *     next to the solid, whose consumed solute precipitates as deposited
 *     mass m; once m reaches a threshold the node turns solid (surface
 *     growth, eventually pore closure).
 *
 * Every step is taken in this order on the whole lattice (one pass each,
 * no fusion, no blocking):
 *   moments -> cohesion + adhesion forces -> Shan-Chen velocity shift ->
 *   BGK collide (A, B) -> D2Q4 collide (inlet column imposed) ->
 *   surface reaction -> stream with bounce-back (push form) ->
 *   deposit + threshold test -> all flagged nodes turn solid at once.
 *
 * Readings taken where the paper is silent (it defers all details to a
 * companion paper) are listed with the function that applies them.
 *
 * Lattice: nx * ny nodes, periodic in x and y, node n = y * nx + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9  /* D2Q9 velocities of each fluid component */
#define QS 4 /* D2Q4 velocities of the solute */

/* D2Q9: rest, 4 axis, 4 diagonal; weights 4/9, 1/9, 1/36. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* D2Q4: +x, +y, -x, -y; weight 1/4 each; sound speed squared 1/2. */
static const int SX[QS] = {1, 0, -1, 0};
static const int SY[QS] = {0, 1, 0, -1};
static const int SOPP[QS] = {2, 3, 0, 1};

/* Model constants (one set per lattice). */
typedef struct {
    double tau_a, tau_b;  /* BGK relaxation times of components A and B */
    double tau_d;         /* BGK relaxation time of the solute, D=(tau_d-1/2)/2 */
    double g_coh;         /* cohesion strength G_c between A and B */
    double g_ads;         /* adhesion g: G_ads,A = -g (A wets), G_ads,B = +g */
    double k_r;           /* reaction-rate constant [lu/ts] */
    double m_threshold;   /* deposited mass at which a node turns solid */
    double c_in;          /* solute concentration imposed at the inlet */
    double body_force_x;  /* uniform acceleration along x (Poiseuille check) */
    int32_t inlet;        /* 1: column x = 0 imposes c_in */
    int32_t cap_x0;       /* capillary section [cap_x0, cap_x1) (closure) */
    int32_t cap_x1;
} orc_params;

typedef struct {
    orc_params p;
    int nx, ny, N;
    double *f;     /* [2][Q][N] post-stream populations of A and B */
    double *g;     /* [QS][N] post-stream solute populations */
    double *m;     /* [N] deposited (precipitated) mass */
    uint8_t *solid;/* [N] 1 = solid */
    /* per-step work arrays */
    double *rho;   /* [2][N] component densities */
    double *j;     /* [2][2][N] component momenta (x, y) */
    double *F;     /* [2][2][N] total force on each component (x, y) */
    double *u;     /* [2][N] barycentric fluid velocity (solute advection) */
    double *fc;    /* [2][Q][N] post-collision A, B */
    double *gc;    /* [QS][N] post-collision solute */
    double *dM;    /* [N] mass precipitated this step */
    uint8_t *flag; /* [N] reached the threshold this step */
    double ledger[4]; /* mass taken out of the fluid by growth: A, B, C, m */
    int64_t step;
    int64_t closure_step; /* first step count with a fully solid column, -1 */
} orc_lattice;

/* Periodic index for a neighbour offset of at most one lattice unit. */
static inline int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

/* BGK equilibrium of D2Q9 (paper Sec. II, "BGK equation"):
 * f_i^eq = w_i rho [1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u]. */
void orc_feq(double rho, double ux, double uy, double *out) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        out[i] = W[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* D2Q4 equilibrium of the solute: g_j^eq = (C/4)(1 + 2 e_j.u). */
void orc_geq(double c, double ux, double uy, double *out) {
    for (int k = 0; k < QS; ++k)
        out[k] = 0.25 * c * (1.0 + 2.0 * (SX[k] * ux + SY[k] * uy));
}

void orc_destroy(orc_lattice *L) {
    if (!L) return;
    free(L->f); free(L->g); free(L->m); free(L->solid);
    free(L->rho); free(L->j); free(L->F); free(L->u);
    free(L->fc); free(L->gc); free(L->dM); free(L->flag);
    free(L);
}

/* Builds a lattice at rest: each fluid node holds the D2Q9 equilibrium at
 * u = 0 for its initial densities rho_a, rho_b and the D2Q4 equilibrium at
 * u = 0 for its initial concentration conc (paper silent on the initial
 * state; rest equilibrium is the reading).  Solid nodes hold nothing. */
orc_lattice *orc_create(const orc_params *p, int nx, int ny,
                        const uint8_t *solid, const double *rho_a,
                        const double *rho_b, const double *conc) {
    if (nx < 1 || ny < 1) return NULL;
    orc_lattice *L = (orc_lattice *)calloc(1, sizeof(orc_lattice));
    if (!L) return NULL;
    L->p = *p;
    L->nx = nx; L->ny = ny; L->N = nx * ny;
    size_t N = (size_t)L->N;
    L->f = (double *)calloc(2 * Q * N, sizeof(double));
    L->g = (double *)calloc(QS * N, sizeof(double));
    L->m = (double *)calloc(N, sizeof(double));
    L->solid = (uint8_t *)calloc(N, 1);
    L->rho = (double *)calloc(2 * N, sizeof(double));
    L->j = (double *)calloc(4 * N, sizeof(double));
    L->F = (double *)calloc(4 * N, sizeof(double));
    L->u = (double *)calloc(2 * N, sizeof(double));
    L->fc = (double *)calloc(2 * Q * N, sizeof(double));
    L->gc = (double *)calloc(QS * N, sizeof(double));
    L->dM = (double *)calloc(N, sizeof(double));
    L->flag = (uint8_t *)calloc(N, 1);
    if (!L->f || !L->g || !L->m || !L->solid || !L->rho || !L->j || !L->F ||
        !L->u || !L->fc || !L->gc || !L->dM || !L->flag) {
        orc_destroy(L);
        return NULL;
    }
    L->closure_step = -1;
    double feq[Q], geq[QS];
    for (size_t n = 0; n < N; ++n) {
        L->solid[n] = solid[n] ? 1 : 0;
        if (L->solid[n]) continue;
        orc_feq(rho_a[n], 0.0, 0.0, feq);
        for (int i = 0; i < Q; ++i) L->f[(0 * Q + i) * N + n] = feq[i];
        orc_feq(rho_b[n], 0.0, 0.0, feq);
        for (int i = 0; i < Q; ++i) L->f[(1 * Q + i) * N + n] = feq[i];
        orc_geq(conc[n], 0.0, 0.0, geq);
        for (int k = 0; k < QS; ++k) L->g[k * N + n] = geq[k];
    }
    /* a section column that is solid from the start: closed at step 0 */
    for (int x = p->cap_x0; x < p->cap_x1 && x < nx && L->closure_step < 0; ++x) {
        int all = 1;
        for (int y = 0; y < ny; ++y)
            if (!L->solid[(size_t)y * nx + x]) { all = 0; break; }
        if (all) L->closure_step = 0;
    }
    return L;
}

/* Moments: component densities and momenta, rho_s = sum_i f_i^s,
 * j_s = sum_i f_i^s e_i.  Solid nodes carry zero density. */
static void moments(orc_lattice *L) {
    size_t N = (size_t)L->N;
    for (size_t n = 0; n < N; ++n) {
        for (int s = 0; s < 2; ++s) {
            double r = 0, jx = 0, jy = 0;
            if (!L->solid[n]) {
                for (int i = 0; i < Q; ++i) {
                    double fi = L->f[(s * Q + i) * N + n];
                    r += fi;
                    jx += fi * EX[i];
                    jy += fi * EY[i];
                }
            }
            L->rho[s * N + n] = r;
            L->j[(s * 2 + 0) * N + n] = jx;
            L->j[(s * 2 + 1) * N + n] = jy;
        }
    }
}

/* Forces: Martys-Chen forces (paper Sec. II, cohesive and adhesive
 * interactions), with D2Q9 weights as the interaction weights:
 *   F_s^coh(x) = -G_c rho_s(x) sum_i w_i rho_s'(x + e_i) e_i   (s' = other)
 *   F_s^ads(x) = -G_ads,s rho_s(x) sum_i w_i solid(x + e_i) e_i
 * with G_ads,A = -g_ads (A attracted to the solid) and G_ads,B = +g_ads.
 * Solid neighbours carry zero density in the cohesion sum.  A uniform body
 * acceleration adds rho_s * body_force_x along x (used only by the
 * Poiseuille check). */
static void forces(orc_lattice *L) {
    size_t N = (size_t)L->N;
    int nx = L->nx, ny = L->ny;
    double Gads[2] = {-L->p.g_ads, +L->p.g_ads};
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            for (int s = 0; s < 2; ++s) {
                double Fx = 0, Fy = 0;
                if (!L->solid[n]) {
                    double cx = 0, cy = 0, ax = 0, ay = 0;
                    for (int i = 1; i < Q; ++i) {
                        size_t nb = (size_t)wrap(y + EY[i], ny) * nx +
                                    wrap(x + EX[i], nx);
                        double rho_other = L->rho[(1 - s) * N + nb];
                        cx += W[i] * rho_other * EX[i];
                        cy += W[i] * rho_other * EY[i];
                        ax += W[i] * L->solid[nb] * EX[i];
                        ay += W[i] * L->solid[nb] * EY[i];
                    }
                    double r = L->rho[s * N + n];
                    Fx = -L->p.g_coh * r * cx - Gads[s] * r * ax +
                         r * L->p.body_force_x;
                    Fy = -L->p.g_coh * r * cy - Gads[s] * r * ay;
                }
                L->F[(s * 2 + 0) * N + n] = Fx;
                L->F[(s * 2 + 1) * N + n] = Fy;
            }
        }
    }
}

/* Collision: Shan-Chen velocity shift and BGK collision of A and B.
 *   u' = sum_s (j_s / tau_s) / sum_s (rho_s / tau_s)
 *   u_s^eq = u' + tau_s F_s / rho_s        (u' when rho_s is ~0)
 *   f_i^s* = f_i^s - (f_i^s - f_i^eq(rho_s, u_s^eq)) / tau_s
 * Also stores the barycentric velocity u = (sum_s j_s + F/2) / sum_s rho_s
 * that advects the solute. */
static void collide_fluid(orc_lattice *L) {
    size_t N = (size_t)L->N;
    double tau[2] = {L->p.tau_a, L->p.tau_b};
    double feq[Q];
    for (size_t n = 0; n < N; ++n) {
        if (L->solid[n]) continue;
        double num_x = 0, num_y = 0, den = 0;
        double jx = 0, jy = 0, Fx = 0, Fy = 0, rt = 0;
        for (int s = 0; s < 2; ++s) {
            num_x += L->j[(s * 2 + 0) * N + n] / tau[s];
            num_y += L->j[(s * 2 + 1) * N + n] / tau[s];
            den += L->rho[s * N + n] / tau[s];
            jx += L->j[(s * 2 + 0) * N + n];
            jy += L->j[(s * 2 + 1) * N + n];
            Fx += L->F[(s * 2 + 0) * N + n];
            Fy += L->F[(s * 2 + 1) * N + n];
            rt += L->rho[s * N + n];
        }
        double upx = den > 0 ? num_x / den : 0.0;
        double upy = den > 0 ? num_y / den : 0.0;
        for (int s = 0; s < 2; ++s) {
            double r = L->rho[s * N + n];
            double ux = upx, uy = upy;
            if (r > 1e-12) {
                ux += tau[s] * L->F[(s * 2 + 0) * N + n] / r;
                uy += tau[s] * L->F[(s * 2 + 1) * N + n] / r;
            }
            orc_feq(r, ux, uy, feq);
            for (int i = 0; i < Q; ++i) {
                double fi = L->f[(s * Q + i) * N + n];
                L->fc[(s * Q + i) * N + n] = fi - (fi - feq[i]) / tau[s];
            }
        }
        L->u[0 * N + n] = rt > 0 ? (jx + 0.5 * Fx) / rt : 0.0;
        L->u[1 * N + n] = rt > 0 ? (jy + 0.5 * Fy) / rt : 0.0;
    }
}

/* Solute collision: BGK collision of the D2Q4 solute, advected by u.  At the inlet
 * column (x = 0, when enabled) the post-collision solute is the
 * equilibrium at c_in and the node's own u (reading of the unstated inlet
 * condition: a Dirichlet concentration imposed at each collision). */
static void collide_solute(orc_lattice *L) {
    size_t N = (size_t)L->N;
    double geq[QS];
    for (size_t n = 0; n < N; ++n) {
        if (L->solid[n]) continue;
        int x = (int)(n % (size_t)L->nx);
        double ux = L->u[n], uy = L->u[N + n];
        if (L->p.inlet && x == 0) {
            orc_geq(L->p.c_in, ux, uy, geq);
            for (int k = 0; k < QS; ++k) L->gc[k * N + n] = geq[k];
            continue;
        }
        double c = 0;
        for (int k = 0; k < QS; ++k) c += L->g[k * N + n];
        orc_geq(c, ux, uy, geq);
        for (int k = 0; k < QS; ++k) {
            double gk = L->g[k * N + n];
            L->gc[k * N + n] = gk - (gk - geq[k]) / L->p.tau_d;
        }
    }
}

/* Surface reaction (paper Sec. II: mass deposits on the surface
 * at a rate set by k_r).  Reading: first order and irreversible; at a fluid
 * node where the wetting melt is the majority (rho_A > rho_B) and that has
 * n_s > 0 solid D2Q4 neighbours, the amount dM = k_r n_s C* leaves the
 * solute (C* = post-collision concentration) by scaling every g_j* by
 * (1 - k_r n_s), clamped at zero, and precipitates at the node. */
static void react(orc_lattice *L) {
    size_t N = (size_t)L->N;
    int nx = L->nx, ny = L->ny;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            L->dM[n] = 0.0;
            if (L->solid[n]) continue;
            if (!(L->rho[n] > L->rho[N + n])) continue;
            int ns = 0;
            for (int k = 0; k < QS; ++k)
                ns += L->solid[(size_t)wrap(y + SY[k], ny) * nx +
                               wrap(x + SX[k], nx)];
            if (ns == 0) continue;
            double cstar = 0;
            for (int k = 0; k < QS; ++k) cstar += L->gc[k * N + n];
            double keep = 1.0 - L->p.k_r * ns;
            if (keep < 0.0) keep = 0.0;
            for (int k = 0; k < QS; ++k) L->gc[k * N + n] *= keep;
            L->dM[n] = cstar * (1.0 - keep);
        }
    }
}

/* Streaming with half-way bounce-back (paper Sec. II, bounce-back
 * rule).  A post-collision population leaving fluid node x along e_i lands
 * at x + e_i if that node is fluid; if it is solid the population returns
 * to x in the opposite direction.  The same rule moves the solute. */
static void stream(orc_lattice *L) {
    size_t N = (size_t)L->N;
    int nx = L->nx, ny = L->ny;
    memset(L->f, 0, 2 * Q * N * sizeof(double));
    memset(L->g, 0, QS * N * sizeof(double));
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            if (L->solid[n]) continue;
            for (int s = 0; s < 2; ++s) {
                for (int i = 0; i < Q; ++i) {
                    double v = L->fc[(s * Q + i) * N + n];
                    size_t d = (size_t)wrap(y + EY[i], ny) * nx +
                               wrap(x + EX[i], nx);
                    if (L->solid[d])
                        L->f[(s * Q + OPP[i]) * N + n] += v;
                    else
                        L->f[(s * Q + i) * N + d] += v;
                }
            }
            for (int k = 0; k < QS; ++k) {
                double v = L->gc[k * N + n];
                size_t d = (size_t)wrap(y + SY[k], ny) * nx +
                           wrap(x + SX[k], nx);
                if (L->solid[d])
                    L->g[SOPP[k] * N + n] += v;
                else
                    L->g[k * N + d] += v;
            }
        }
    }
}

/* Deposit and growth: the precipitated mass accumulates, m += dM; every fluid
 * node with m >= m_threshold turns solid (paper Sec. II: the solid phase
 * expands once the cumulated mass exceeds a threshold).  Reading: all
 * nodes flagged in a step turn solid together after streaming; their
 * fluid (A, B), solute and deposit go to the growth ledger and their
 * populations are cleared; nothing is passed to neighbours.  The first
 * step count at which some column of the capillary section is entirely
 * solid is the pore-closure step. */
static void deposit_and_grow(orc_lattice *L) {
    size_t N = (size_t)L->N;
    int nx = L->nx, ny = L->ny;
    int any = 0;
    for (size_t n = 0; n < N; ++n) {
        L->flag[n] = 0;
        if (L->solid[n]) continue;
        L->m[n] += L->dM[n];
        if (L->m[n] >= L->p.m_threshold) {
            L->flag[n] = 1;
            any = 1;
        }
    }
    if (!any) return;
    for (size_t n = 0; n < N; ++n) {
        if (!L->flag[n]) continue;
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < Q; ++i) {
                L->ledger[s] += L->f[(s * Q + i) * N + n];
                L->f[(s * Q + i) * N + n] = 0.0;
            }
        for (int k = 0; k < QS; ++k) {
            L->ledger[2] += L->g[k * N + n];
            L->g[k * N + n] = 0.0;
        }
        L->ledger[3] += L->m[n];
        L->m[n] = 0.0;
        L->solid[n] = 1;
    }
    if (L->closure_step < 0) {
        for (int x = L->p.cap_x0; x < L->p.cap_x1 && x < nx; ++x) {
            int all = 1;
            for (int y = 0; y < ny; ++y)
                if (!L->solid[(size_t)y * nx + x]) { all = 0; break; }
            if (all) { L->closure_step = L->step + 1; break; }
        }
    }
}

void orc_step(orc_lattice *L, int64_t nsteps) {
    for (int64_t t = 0; t < nsteps; ++t) {
        moments(L);
        forces(L);
        collide_fluid(L);
        collide_solute(L);
        react(L);
        stream(L);
        deposit_and_grow(L);
        L->step += 1;
    }
}

/* ---- accessors used by the Python wrapper --------------------------- */

int orc_nx(const orc_lattice *L) { return L->nx; }
int orc_ny(const orc_lattice *L) { return L->ny; }
int64_t orc_step_count(const orc_lattice *L) { return L->step; }
int64_t orc_closure_step(const orc_lattice *L) { return L->closure_step; }
void orc_ledger(const orc_lattice *L, double *out4) {
    for (int k = 0; k < 4; ++k) out4[k] = L->ledger[k];
}

/* which: 0 = populations f (2*Q*N: A then B, direction-major),
 *        1 = solute g (QS*N), 2 = deposit m (N). */
int orc_get(const orc_lattice *L, int which, double *out) {
    size_t N = (size_t)L->N;
    switch (which) {
    case 0: memcpy(out, L->f, 2 * Q * N * sizeof(double)); return 0;
    case 1: memcpy(out, L->g, QS * N * sizeof(double)); return 0;
    case 2: memcpy(out, L->m, N * sizeof(double)); return 0;
    default: return -1;
    }
}

int orc_set(orc_lattice *L, int which, const double *in) {
    size_t N = (size_t)L->N;
    switch (which) {
    case 0: memcpy(L->f, in, 2 * Q * N * sizeof(double)); return 0;
    case 1: memcpy(L->g, in, QS * N * sizeof(double)); return 0;
    case 2: memcpy(L->m, in, N * sizeof(double)); return 0;
    default: return -1;
    }
}

void orc_get_solid(const orc_lattice *L, uint8_t *out) {
    memcpy(out, L->solid, (size_t)L->N);
}

/* Densities (2*N) and forces (2 components x 2 axes x N) of the current
 * post-stream state, exactly as the next step would use them. */
void orc_moments_forces(orc_lattice *L, double *rho_out, double *F_out) {
    size_t N = (size_t)L->N;
    moments(L);
    forces(L);
    memcpy(rho_out, L->rho, 2 * N * sizeof(double));
    memcpy(F_out, L->F, 4 * N * sizeof(double));
}
