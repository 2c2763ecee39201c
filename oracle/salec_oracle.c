/*
 * salec_oracle.c -- serial FP64 CPU oracle of the SALEc-2D explicit time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg use it, through oracle/oracle.py.  It shares no code with the CUDA library.
 *
 * What it computes: one SALE cycle (Amsden et al. 1980, which the paper cites for its
 * operator split, Sect. 2) on a 2D axisymmetric Eulerian grid:
 *   phase 0  equation of state, artificial viscosity and the Courant time step (Sect. 6, Eq. 14)
 *   phase 1  Lagrangian momentum, Eq. 1, with the PML stress-auxiliary psi1 (Sect. 3, Eqs. 16-17)
 *   phase 2  Lagrangian energy, Eq. 2, strength and damage, PML psi2
 *   phase 3  Eulerian donor-cell remap, Eqs. 3-5, with the PML phi1..phi3 and the damping
 *            terms of the PML control equations (Sect. 3, Eqs. 23-25)
 * The discrete choices the paper leaves open (staggering, corner forces, void rules,
 * remap, PML discretisation, boundary conditions) follow the written readings of the
 * scheme; every function below says which step it is.  Everything is plain FP64 with
 * full-grid arrays and straight loops, built with -O2 -ffp-contract=off.
 *
 * Parity status of each function is stated next to it: "pinned by <test>" names the
 * closed form or invariant in tests/test_oracle_*.py that checks it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXMAT 3

enum { ORC_EOS_TILLOTSON = 0, ORC_EOS_IDEAL_GAS = 1 };
enum { ORC_STR_NONE = 0, ORC_STR_COLLINS = 1 };
enum { ORC_TOP_OUTFLOW = 0, ORC_TOP_WALL = 1 };
enum { ORC_BOTTOM_NOSLIP = 0, ORC_BOTTOM_FREESLIP = 1 };

typedef struct {
    int eos;                 /* ORC_EOS_* */
    double rho0;             /* reference density */
    double A, B, E0, a, b, alpha, beta, Eiv, Ecv;   /* Tillotson constants */
    double gamma;            /* ideal gas */
    int strength;            /* ORC_STR_* */
    double Yi0, mui, Yim, Yd0, mud, Ydm;            /* Collins et al. 2004 yield surfaces */
    double G;                /* shear modulus */
    double eps_fb, B_dam, p_bd;                     /* failure strain eps_f = max(eps_fb, B_dam (p - p_bd)) */
    double p_t;              /* tensile limit of intact material (<= 0) */
} orc_material;

typedef struct {
    int nr, nz, nmat;
    double dx;
    int pml_r, pml_b;
    double pml_R, pml_c, pml_alpha;
    double gravity, cfl, dt_init, dt_max, dt_growth, dt_min;
    double av_cq, av_cl, f_min;
    int bc_top, bc_bottom;
} orc_grid;

typedef struct {
    orc_grid g;
    orc_material mat[ORC_MAXMAT];
    int ncell, nvert;
    /* geometry (per radian): column widths dr[i], vertex radii rR[i] (nr+1), centre radii
       rc[i] = (r_i + r_i+1) / 2 and vertical face areas A_Z[i] = rc dr; row heights dz[j]
       and vertex heights zv[j] (nz+1).  The radial face at r_i of row j has area
       rR[i] dz[j]; cell (i,j) has volume A_Z[i] dz[j]. */
    double *dr, *rR, *rc, *A_Z, *dz, *zv;
    int has_content;                     /* a layer or projectile is in: the spacing is fixed */
    /* state */
    double *f[ORC_MAXMAT], *rho[ORC_MAXMAT], *I, *srr, *szz, *srz, *D, *pmax;
    double *vr, *vz;
    /* PML auxiliaries, full-grid arrays (zero outside the strips) */
    double *phi1_b, *phi3_b, *psi2_b, *phi1_r, *phi3_r, *psi2_r;      /* cells */
    double *phi2r_b, *phi2z_b, *psi1r_b, *psi1z_b;                     /* vertices, bottom strip */
    double *phi2r_r, *phi2z_r, *psi1r_r, *psi1z_r;                     /* vertices, right strip */
    double *dB_c, *dB_v, *dR_c, *dR_v;   /* damping profiles: rows (cells, vertices), columns */
    double *wR_c, *wR_v;                 /* 1 on rows whose reference state holds material (cells, vertices) */
    double alpha_b, alpha_r;             /* relaxation rates of the strips' auxiliaries */
    double *p0, *rho_ref, *I_ref;        /* reference state per row */
    /* set-up accumulators */
    double *setup_V[ORC_MAXMAT], *setup_M[ORC_MAXMAT], *setup_E, *setup_Pz;
    double *setup_R[ORC_MAXMAT], *setup_mix[ORC_MAXMAT];   /* density of the contributions; 1 if they differ */
    double *setup_I, *setup_Imix;                          /* likewise for the specific energy */
    double *hyd_P, *hyd_R;               /* rows set by a hydrostatic layer: their pressure and density */
    int finalized;
    /* scalars */
    double t, dt, dt_prev;
    long nstep;
    double mass_out, zmom_out, ie_out, mass_discarded, mass_pml;
    double ke_lag, ie_lag;   /* kinetic and internal energy right after the Lagrangian phase */
    int status;
    /* per-step work arrays */
    double *P, *pbar, *mv, *vLr, *vLz, *dK, *kheat;
    double *VL, *fL[ORC_MAXMAT], *rhoL[ORC_MAXMAT], *IL, *srrL, *szzL, *srzL, *DL;
    double *dVR, *dVZ, *dMR, *dMZ;
} orc_sim;

#define CID(s, i, j) ((j) * (s)->g.nr + (i))
#define VID(s, i, j) ((j) * ((s)->g.nr + 1) + (i))

/* radial face at r_i of row j, volume of cell (i,j), and the cell's length scale (its
   smaller side) for the viscosity and the Courant condition */
static double face_r(const orc_sim* s, int i, int j) { return s->rR[i] * s->dz[j]; }
static double vol(const orc_sim* s, int i, int j) { return s->A_Z[i] * s->dz[j]; }
static double cell_len(const orc_sim* s, int i, int j) { return s->dr[i] < s->dz[j] ? s->dr[i] : s->dz[j]; }

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* ------------------------------------------------------------------------------------
 * Equations of state.  The paper inherits its EoS from SALEc ("various equations of
 * state", Sect. 1; "inherited from SALEc", Sect. 2); the hot path uses Tillotson (1962).
 * Returns the unclipped pressure and the squared sound speed
 *   c^2 = dp/drho|_I + (p / rho^2) dp/dI|_rho.
 * Pinned by test_oracle_eos.py (reference-state zero, bulk sound speed A/rho0, Grueneisen
 * limits a+b and a, ideal-gas limit at vanishing density, continuity at rho0 and at the
 * blend ends, derivatives against central differences).
 * ------------------------------------------------------------------------------------ */
static void tillotson(const orc_material* m, double rho_in, double I_in, double* p_out, double* c2_out)
{
    double I = I_in > 0.0 ? I_in : 0.0;
    /* evaluated at no less than rho_f = 1e-12 rho0 (reading): there the form is in its
       dilute limit, where c^2 no longer depends on rho and the pressure is proportional to
       it (p = a rho I once the exponential terms vanish), so below rho_f the pressure at
       rho_f is scaled back by rho / rho_f and c^2 is taken at rho_f; the floor keeps the
       rho^-2 terms finite in FP32 as well */
    const double rho_f = 1e-12 * m->rho0;
    double rho = rho_in > rho_f ? rho_in : rho_f;
    double eta = rho / m->rho0;
    double mu = eta - 1.0;
    double w0 = I / (m->E0 * eta * eta) + 1.0;
    /* compressed branch p_c */
    double pc = (m->a + m->b / w0) * rho * I + m->A * mu + m->B * mu * mu;
    double dpc_drho = (m->a + m->b / w0) * I + 2.0 * m->b * I * I / (w0 * w0 * m->E0 * eta * eta)
                      + (m->A + 2.0 * m->B * mu) / m->rho0;
    double dpc_dI = rho * (m->a + m->b / w0 - m->b * I / (w0 * w0 * m->E0 * eta * eta));
    double p, c2;
    if (rho >= m->rho0 || I <= m->Eiv) {
        p = pc;
        c2 = dpc_drho + pc / (rho * rho) * dpc_dI;
    } else {
        /* expanded branch p_e */
        double x = m->rho0 / rho - 1.0;
        double Ea = exp(-m->alpha * x * x);
        double Eb = exp(-m->beta * x);
        double dx_drho = -m->rho0 / (rho * rho);
        double bterm = m->b * rho * I / w0;
        double dbterm_drho = m->b * I / w0 + 2.0 * m->b * I * I / (w0 * w0 * m->E0 * eta * eta);
        double aterm = m->A * mu * Eb;
        double daterm_drho = (m->A / m->rho0) * Eb + m->A * mu * Eb * (-m->beta) * dx_drho;
        double pe = m->a * rho * I + (bterm + aterm) * Ea;
        double dpe_drho = m->a * I + (dbterm_drho + daterm_drho) * Ea
                          + (bterm + aterm) * Ea * (-2.0 * m->alpha * x) * dx_drho;
        double dpe_dI = m->a * rho + (m->b * rho / w0 - m->b * rho * I / (w0 * w0 * m->E0 * eta * eta)) * Ea;
        const double ce2 = dpe_drho + pe / (rho * rho) * dpe_dI;
        if (I >= m->Ecv) {
            p = pe;
            c2 = ce2;
        } else {
            /* linear blend in I between the two branches; the sound speed is the same blend
               of the branches' own sound speeds (reading: the derivative of the blended
               pressure adds (p_e - p_c)/(E_cv - E_iv) p/rho^2, which grows without bound
               as rho -> 0 when A != B and is discontinuous at both blend ends) */
            double den = m->Ecv - m->Eiv;
            double we = I - m->Eiv, wc = m->Ecv - I;
            p = (we * pe + wc * pc) / den;
            const double cc2 = dpc_drho + pc / (rho * rho) * dpc_dI;
            c2 = (we * ce2 + wc * cc2) / den;
        }
    }
    /* a near-empty cell keeps the dilute gas's pressure, not the one at rho_f: its pressure
       gradient per unit mass stays ~ a I / dx */
    if (rho_in < rho_f) p = p * ((rho_in > 0.0 ? rho_in : 0.0) / rho_f);
    double floor2 = 0.01 * m->A / m->rho0;
    if (!(c2 > floor2)) c2 = floor2;
    *p_out = p;
    *c2_out = c2;
}

/* Ideal gas, p = (gamma - 1) rho I: the equation of state of the Sod shock-tube pin. */
static void ideal_gas(const orc_material* m, double rho, double I_in, double* p_out, double* c2_out)
{
    double I = I_in > 0.0 ? I_in : 0.0;
    *p_out = (m->gamma - 1.0) * rho * I;
    *c2_out = m->gamma * (m->gamma - 1.0) * I;
}

static void material_eos(const orc_material* m, double rho, double I, double* p, double* c2)
{
    if (m->eos == ORC_EOS_IDEAL_GAS) ideal_gas(m, rho, I, p, c2);
    else tillotson(m, rho, I, p, c2);
}

/* ------------------------------------------------------------------------------------
 * Strength and tension of strongly expanded material.  Reading: rock expanded well below
 * its reference density is fragmented; below rho0 / 2 it carries neither shear strength
 * nor tension, and between rho0 / 2 and rho0 both are scaled by w = 2 rho / rho0 - 1.  In
 * dilute ejecta (1e-7 of rho0 and less) a stress or tension of even the damaged cohesion
 * times the strain of a step, per unit of so little mass, sends the specific energy to
 * +-1e10 J/kg.  Pinned by test_oracle_strength.py.
 * ------------------------------------------------------------------------------------ */
static double expansion_weight(const orc_material* m, double rho)
{
    double w = 2.0 * rho / m->rho0 - 1.0;
    return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
}

/* ------------------------------------------------------------------------------------
 * Collins et al. (2004) pressure-dependent yield strength (Sect. 1 cites it; Table 1
 * lists its constants), blended by the scalar damage D:
 *   Y_i = Y_i0 + mu_i p / (1 + mu_i p / (Y_im - Y_i0)),  Y_d = min(Y_d0 + mu_d p, Y_dm),
 *   Y = (1 - D) Y_i + D Y_d, evaluated at max(p, 0), times the thermal-softening factor
 *   below (1 at I = 0) and the expansion weight above (1 at rho >= rho0).
 * Pinned by test_oracle_strength.py (limits p -> 0, p -> infinity, D = 0 and D = 1;
 * softening factor tanh(1.2) at I = E_iv / 2, zero from E_iv up).
 * ------------------------------------------------------------------------------------ */
static double collins_yield(const orc_material* m, double p_in, double D, double I, double rho)
{
    double p = p_in > 0.0 ? p_in : 0.0;
    double Yi = m->Yi0 + m->mui * p / (1.0 + m->mui * p / (m->Yim - m->Yi0));
    double Yd = m->Yd0 + m->mud * p;
    if (Yd > m->Ydm) Yd = m->Ydm;
    double Y = (1.0 - D) * Yi + D * Yd;
    /* thermal softening (Collins et al. 2004): Y tanh(xi (T_m / T - 1)), xi = 1.2, zero at
       and above melting.  The state carries no temperature; reading: T_m / T = E_iv / I with
       the Tillotson incipient-vaporisation energy as the melt-energy scale */
    if (I > 0.0) {
        if (!(I < m->Eiv)) return 0.0;
        Y *= tanh(1.2 * (m->Eiv / I - 1.0));
    }
    Y *= expansion_weight(m, rho);
    return Y > 0.0 ? Y : 0.0;
}

/* ------------------------------------------------------------------------------------
 * PML attenuation profile, Sect. 3 Eq. 26: d(y) = 3c/(2 delta) (y/delta)^2 ln(1/R),
 * y measured from the inner edge of the strip, delta = width * dx.
 * Pinned by test_oracle_pml.py (round-trip attenuation exp(-2 int d/c) = R).
 * ------------------------------------------------------------------------------------ */
static double pml_profile(double c, double width_cells, double dx, double y_cells, double R)
{
    if (width_cells <= 0.0 || y_cells <= 0.0) return 0.0;
    double delta = width_cells * dx;
    double s = y_cells / width_cells;
    return 1.5 * c / delta * s * s * log(1.0 / R);
}

/* The same profile with the strip's thickness delta and the distance y in metres (a
   strip of cells of any heights). */
static double pml_profile_len(double c, double delta, double y, double R)
{
    double s = y / delta;
    return 1.5 * c / delta * s * s * log(1.0 / R);
}

/* Vertex positions, centre radii and face areas from the cell sizes, summed outward from
   the axis and up from the bottom. */
static void set_geometry(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz;
    s->rR[0] = 0.0;
    for (int i = 0; i < nr; ++i) s->rR[i + 1] = s->rR[i] + s->dr[i];
    for (int i = 0; i < nr; ++i) {
        s->rc[i] = 0.5 * (s->rR[i] + s->rR[i + 1]);
        s->A_Z[i] = s->rc[i] * s->dr[i];
    }
    s->zv[0] = 0.0;
    for (int j = 0; j < nz; ++j) s->zv[j + 1] = s->zv[j] + s->dz[j];
}

/* ------------------------------------------------------------------------------------ */
orc_sim* orc_create(const orc_grid* g, const orc_material* mats)
{
    if (g->nr < 1 || g->nz < 1 || g->nmat < 1 || g->nmat > ORC_MAXMAT || !(g->dx > 0.0)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->g = *g;
    for (int m = 0; m < g->nmat; ++m) s->mat[m] = mats[m];
    int nr = g->nr, nz = g->nz;
    s->ncell = nr * nz;
    s->nvert = (nr + 1) * (nz + 1);
    s->dr = zalloc(nr); s->rR = zalloc(nr + 1); s->rc = zalloc(nr); s->A_Z = zalloc(nr);
    s->dz = zalloc(nz); s->zv = zalloc(nz + 1);
    for (int i = 0; i < nr; ++i) s->dr[i] = g->dx;      /* uniform until orc_set_spacing */
    for (int j = 0; j < nz; ++j) s->dz[j] = g->dx;
    set_geometry(s);
    size_t nc = s->ncell, nv = s->nvert;
    for (int m = 0; m < ORC_MAXMAT; ++m) {
        s->f[m] = zalloc(nc); s->rho[m] = zalloc(nc);
        s->fL[m] = zalloc(nc); s->rhoL[m] = zalloc(nc);
        s->setup_V[m] = zalloc(nc); s->setup_M[m] = zalloc(nc);
        s->setup_R[m] = zalloc(nc); s->setup_mix[m] = zalloc(nc);
    }
    s->I = zalloc(nc); s->srr = zalloc(nc); s->szz = zalloc(nc); s->srz = zalloc(nc);
    s->D = zalloc(nc); s->pmax = zalloc(nc);
    s->vr = zalloc(nv); s->vz = zalloc(nv);
    s->phi1_b = zalloc(nc); s->phi3_b = zalloc(nc); s->psi2_b = zalloc(nc);
    s->phi1_r = zalloc(nc); s->phi3_r = zalloc(nc); s->psi2_r = zalloc(nc);
    s->phi2r_b = zalloc(nv); s->phi2z_b = zalloc(nv); s->psi1r_b = zalloc(nv); s->psi1z_b = zalloc(nv);
    s->phi2r_r = zalloc(nv); s->phi2z_r = zalloc(nv); s->psi1r_r = zalloc(nv); s->psi1z_r = zalloc(nv);
    s->dB_c = zalloc(nz); s->dB_v = zalloc(nz + 1); s->dR_c = zalloc(nr); s->dR_v = zalloc(nr + 1);
    s->wR_c = zalloc(nz); s->wR_v = zalloc(nz + 1);
    s->p0 = zalloc(nz); s->rho_ref = zalloc(nz); s->I_ref = zalloc(nz);
    s->setup_E = zalloc(nc); s->setup_Pz = zalloc(nc); s->setup_I = zalloc(nc); s->setup_Imix = zalloc(nc);
    s->hyd_P = zalloc(nz); s->hyd_R = zalloc(nz);
    s->P = zalloc(nc); s->pbar = zalloc(nc); s->mv = zalloc(nv); s->vLr = zalloc(nv); s->vLz = zalloc(nv);
    s->dK = zalloc(nv); s->kheat = zalloc(nv);
    s->VL = zalloc(nc); s->IL = zalloc(nc); s->srrL = zalloc(nc); s->szzL = zalloc(nc); s->srzL = zalloc(nc);
    s->DL = zalloc(nc);
    s->dVR = zalloc((size_t)(nr + 1) * nz); s->dVZ = zalloc((size_t)nr * (nz + 1));
    s->dMR = zalloc((size_t)(nr + 1) * nz); s->dMZ = zalloc((size_t)nr * (nz + 1));
    s->dt_prev = g->dt_init;
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    double** all[] = {&s->dr, &s->rR, &s->rc, &s->A_Z, &s->dz, &s->zv, &s->I, &s->srr, &s->szz, &s->srz, &s->D, &s->pmax,
                      &s->vr, &s->vz, &s->phi1_b, &s->phi3_b, &s->psi2_b, &s->phi1_r, &s->phi3_r,
                      &s->psi2_r, &s->phi2r_b, &s->phi2z_b, &s->psi1r_b, &s->psi1z_b, &s->phi2r_r,
                      &s->phi2z_r, &s->psi1r_r, &s->psi1z_r, &s->dB_c, &s->dB_v, &s->dR_c, &s->dR_v, &s->wR_c, &s->wR_v,
                      &s->p0, &s->rho_ref, &s->I_ref, &s->setup_E, &s->setup_Pz, &s->setup_I, &s->setup_Imix, &s->hyd_P, &s->hyd_R, &s->P, &s->pbar,
                      &s->mv, &s->vLr, &s->vLz, &s->dK, &s->kheat, &s->VL, &s->IL, &s->srrL, &s->szzL, &s->srzL, &s->DL,
                      &s->dVR, &s->dVZ, &s->dMR, &s->dMZ};
    for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); ++k) free(*all[k]);
    for (int m = 0; m < ORC_MAXMAT; ++m) {
        free(s->f[m]); free(s->rho[m]); free(s->fL[m]); free(s->rhoL[m]);
        free(s->setup_V[m]); free(s->setup_M[m]); free(s->setup_R[m]); free(s->setup_mix[m]);
    }
    free(s);
}

/* ------------------------------------------------------------------------------------
 * Initial conditions.  A layer fills rows between two heights; a projectile is a sphere
 * on the symmetry axis whose cell fractions are r-weighted 16x16 sub-samples.  With
 * gravity a cold Tillotson layer (rho <= 0 requested) is put in discrete hydrostatic
 * equilibrium, -grad p0 + rho g = 0 (Sect. 3, the constraint on p0), solved per row by
 * Newton's method from the surface down.  Layers stack: a hydrostatic layer whose top row
 * lies right below a row of an earlier hydrostatic layer starts from that row's pressure
 * and density (its overburden), so a layered target (the paper's sediment / crust / mantle
 * column, Sect. 4) is built from the top down.  Pinned by test_oracle_rest.py (hydrostatic
 * columns, single and stacked, stay at rest; the stacked column's pressure matches the
 * overburden) and test_oracle_setup.py (sphere volume).
 * ------------------------------------------------------------------------------------ */
/* one contribution of material `mat` to cell c; a cell whose contributions all share one
   density keeps that density exactly (M / V would round it) */
static void contribute(orc_sim* s, int mat, int c, double vol, double rho, double I0, double vz)
{
    double mass = rho * vol;
    int empty = 1;
    for (int m = 0; m < s->g.nmat; ++m) if (s->setup_V[m][c] != 0.0) empty = 0;
    if (empty) s->setup_I[c] = I0;
    else if (s->setup_I[c] != I0) s->setup_Imix[c] = 1.0;
    if (s->setup_V[mat][c] == 0.0) s->setup_R[mat][c] = rho;
    else if (s->setup_R[mat][c] != rho) s->setup_mix[mat][c] = 1.0;
    s->setup_V[mat][c] += vol;
    s->setup_M[mat][c] += mass;
    s->setup_E[c] += mass * I0;
    s->setup_Pz[c] += mass * vz;
}

/* Non-uniform cells: widths dr[nr] and heights dz[nz] (m, positive), before any layer or
   projectile.  The paper's grids have a high-resolution zone of equal cells and extension
   zones whose cells grow geometrically (Table 2: factor 1.05 up to a maximum spacing). */
int orc_set_spacing(orc_sim* s, const double* dr, const double* dz)
{
    if (s->finalized || s->has_content) return 1;
    for (int i = 0; i < s->g.nr; ++i) if (!(dr[i] > 0.0)) return 2;
    for (int j = 0; j < s->g.nz; ++j) if (!(dz[j] > 0.0)) return 2;
    for (int i = 0; i < s->g.nr; ++i) s->dr[i] = dr[i];
    for (int j = 0; j < s->g.nz; ++j) s->dz[j] = dz[j];
    set_geometry(s);
    return 0;
}

int orc_add_layer(orc_sim* s, int mat, double zlo, double zhi, double rho, double I0, double vz)
{
    if (s->finalized || mat < 0 || mat >= s->g.nmat || !(zhi > zlo)) return 1;
    const orc_material* m = &s->mat[mat];
    int nr = s->g.nr, nz = s->g.nz;
    int hydro = (rho <= 0.0 && s->g.gravity > 0.0 && m->eos == ORC_EOS_TILLOTSON);
    if (hydro && I0 != 0.0) return 1;
    s->has_content = 1;
    /* overlap fraction of each row */
    double* w = zalloc(nz);
    for (int j = 0; j < nz; ++j) {
        double z0 = s->zv[j], z1 = s->zv[j + 1];
        double lo = zlo > z0 ? zlo : z0, hi = zhi < z1 ? zhi : z1;
        /* a row inside the layer is full (z1 - z0 need not round to dz exactly) */
        w[j] = (zlo <= z0 && zhi >= z1) ? 1.0 : (hi > lo ? (hi - lo) / s->dz[j] : 0.0);
    }
    double* rowrho = zalloc(nz);
    if (!hydro) {
        double r = rho > 0.0 ? rho : m->rho0;
        for (int j = 0; j < nz; ++j) rowrho[j] = r;
    } else {
        /* rows must be completely filled or empty; walk down from the top filled row.
           Balance at the vertex between row j (below) and row j+1 (above):
           P_j - P_{j+1} = g (rho_j dz_j + rho_{j+1} dz_{j+1}) / 2, with P_j = A mu + B mu^2
           (I = 0).  Wabove = g rho_{j+1} dz_{j+1} / 2, the upper half cell's weight. */
        double Pabove = 0.0, Wabove = 0.0;
        int top = -1;
        for (int j = nz - 1; j >= 0; --j) if (w[j] > 0.0) { top = j; break; }
        for (int j = 0; j < nz; ++j)
            if (w[j] > 0.0 && w[j] < 1.0) { free(w); free(rowrho); return 2; }
        /* overburden: the row right above, if an earlier hydrostatic layer filled it */
        if (top >= 0 && top + 1 < nz && s->hyd_R[top + 1] > 0.0) {
            Pabove = s->hyd_P[top + 1];
            Wabove = (0.5 * s->dz[top + 1] * s->g.gravity) * s->hyd_R[top + 1];
        }
        for (int j = top; j >= 0 && w[j] > 0.0; --j) {
            double k = 0.5 * s->dz[j] * s->g.gravity;
            double rhs = Pabove + Wabove;
            double mu = 0.0;
            for (int it = 0; it < 100; ++it) {
                double r = m->rho0 * (1.0 + mu);
                double fval = m->A * mu + m->B * mu * mu - k * r - rhs;
                double fder = m->A + 2.0 * m->B * mu - k * m->rho0;
                double step = fval / fder;
                mu -= step;
                if (fabs(step) <= 1e-17 * (1.0 + fabs(mu))) break;
            }
            rowrho[j] = m->rho0 * (1.0 + mu);
            Pabove = m->A * mu + m->B * mu * mu;
            Wabove = k * rowrho[j];
            s->hyd_P[j] = Pabove;
            s->hyd_R[j] = rowrho[j];
        }
    }
    for (int j = 0; j < nz; ++j) {
        if (w[j] <= 0.0) continue;
        for (int i = 0; i < nr; ++i) {
            contribute(s, mat, CID(s, i, j), w[j] * vol(s, i, j), rowrho[j], I0, vz);
        }
    }
    free(w); free(rowrho);
    return 0;
}

int orc_place_projectile(orc_sim* s, int mat, double radius, double zc, double vz, double rho, double I0)
{
    if (s->finalized || mat < 0 || mat >= s->g.nmat || !(radius > 0.0)) return 1;
    const orc_material* m = &s->mat[mat];
    double r = rho > 0.0 ? rho : m->rho0;
    int nr = s->g.nr, nz = s->g.nz;
    s->has_content = 1;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            double inside = 0.0, total = 0.0;
            for (int b = 0; b < 16; ++b) {
                for (int a = 0; a < 16; ++a) {
                    double rs = s->rR[i] + s->dr[i] * (((double)a + 0.5) / 16.0);
                    double zs = s->zv[j] + s->dz[j] * (((double)b + 0.5) / 16.0);
                    double dz = zs - zc;
                    total += rs;
                    if (rs * rs + dz * dz < radius * radius) inside += rs;
                }
            }
            double frac = inside / total;
            if (frac <= 0.0) continue;
            int c = CID(s, i, j);
            /* the projectile displaces layer material */
            double keep = 1.0 - frac;
            for (int k = 0; k < s->g.nmat; ++k) {
                s->setup_V[k][c] *= keep;
                s->setup_M[k][c] *= keep;
            }
            s->setup_E[c] *= keep;
            s->setup_Pz[c] *= keep;
            contribute(s, mat, c, frac * vol(s, i, j), r, I0, vz);
        }
    }
    return 0;
}

/* cell matter pressure p_bar = sum_m f_m p_m / sum_m f_m with the tension cutoff; used at
   set-up for the reference state and in phase 0 */
static void cell_eos(const orc_sim* s, int c, double* phat, double* phi, double* c2max, double* rhobar)
{
    double ph = 0.0, fsum = 0.0, c2m = 0.0, mass = 0.0;
    for (int m = 0; m < s->g.nmat; ++m) {
        double fm = s->f[m][c];
        if (!(fm > 0.0)) continue;
        double p, c2;
        material_eos(&s->mat[m], s->rho[m][c], s->I[c], &p, &c2);
        double pmin = (1.0 - s->D[c]) * s->mat[m].p_t * expansion_weight(&s->mat[m], s->rho[m][c]);
        if (p < pmin) p = pmin;
        ph += fm * p;
        fsum += fm;
        mass += fm * s->rho[m][c];
        if (c2 > c2m) c2m = c2;
    }
    *phat = ph;
    *phi = fsum;
    *c2max = c2m;
    *rhobar = fsum > 0.0 ? mass / fsum : 0.0;
}

int orc_finalize(orc_sim* s)
{
    if (s->finalized) return 1;
    int nr = s->g.nr, nz = s->g.nz;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            int c = CID(s, i, j);
            double Mtot = 0.0;
            for (int m = 0; m < s->g.nmat; ++m) {
                double fm = s->setup_V[m][c] / vol(s, i, j);
                if (fm < s->g.f_min) fm = 0.0;
                s->f[m][c] = fm;
                s->rho[m][c] = fm > 0.0 ? (s->setup_mix[m][c] != 0.0 ? s->setup_M[m][c] / s->setup_V[m][c]
                                                                     : s->setup_R[m][c]) : 0.0;
                if (fm > 0.0) Mtot += s->setup_M[m][c];
            }
            s->I[c] = Mtot > 0.0 ? (s->setup_Imix[c] != 0.0 ? s->setup_E[c] / Mtot : s->setup_I[c]) : 0.0;
        }
    }
    /* vertex velocity: quarter-cell momentum over quarter-cell mass */
    for (int j = 0; j <= nz; ++j) {
        for (int i = 0; i <= nr; ++i) {
            double mom = 0.0, mass = 0.0;
            for (int dj = -1; dj <= 0; ++dj) {
                for (int di = -1; di <= 0; ++di) {
                    int ci = i + di, cj = j + dj;
                    if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                    int c = CID(s, ci, cj);
                    double Mc = 0.0, Mall = 0.0;
                    for (int m = 0; m < s->g.nmat; ++m) {
                        Mall += s->setup_M[m][c];
                        if (s->f[m][c] > 0.0) Mc += s->setup_M[m][c];
                    }
                    if (Mall > 0.0) mom += 0.25 * s->setup_Pz[c] * (Mc / Mall);
                    mass += 0.25 * Mc;
                }
            }
            int v = VID(s, i, j);
            s->vr[v] = 0.0;
            s->vz[v] = mass > 0.0 ? mom / mass : 0.0;
            if (j == 0) s->vz[v] = 0.0;
            if (j == nz && s->g.bc_top == ORC_TOP_WALL) s->vz[v] = 0.0;
        }
    }
    /* reference state per row from the outermost column: rho_ref, I_ref and p0 */
    for (int j = 0; j < nz; ++j) {
        int c = CID(s, nr - 1, j);
        double phat, phi, c2, rb;
        cell_eos(s, c, &phat, &phi, &c2, &rb);
        s->rho_ref[j] = rb;
        s->I_ref[j] = phi > 0.0 ? s->I[c] : 0.0;
        s->p0[j] = phi > 0.0 ? phat / phi : 0.0;
    }
    /* PML profiles */
    double c = s->g.pml_c;
    if (!(c > 0.0)) {
        c = 0.0;
        for (int m = 0; m < s->g.nmat; ++m)
            if (s->mat[m].eos == ORC_EOS_TILLOTSON) {
                double cm = sqrt(s->mat[m].A / s->mat[m].rho0);
                if (cm > c) c = cm;
            }
    }
    int pb = s->g.pml_b, pr = s->g.pml_r;
    if ((pb > 0 || pr > 0) && !(c > 0.0 && s->g.pml_R > 0.0 && s->g.pml_R < 1.0)) return 3;
    /* relaxation of the auxiliaries (reading): each auxiliary decays at rate
       alpha = pml_alpha c / delta of its strip, the complex-frequency-shifted stretch
       s = 1 + d / (alpha + i omega) (Kuzuoglu & Mittra 1996) in place of 1 + d / (i omega).
       Without it an auxiliary integrates a static tangential term -- the residual
       deviatoric stress a shock leaves in a strong target -- without bound, and the
       resulting force lifts the bottom strip until a cell empties (a batched impact at
       t = 9 s).  Waves with omega >> alpha are absorbed and passed tangentially as before. */
    /* strips of pb rows and pr columns: thickness delta in metres, y measured from the
       strip's inner edge to the cell centre or vertex */
    const double delta_b = s->zv[pb], r_in = s->rR[nr - pr], delta_r = s->rR[nr] - r_in;
    s->alpha_b = pb > 0 ? s->g.pml_alpha * c / delta_b : 0.0;
    s->alpha_r = pr > 0 ? s->g.pml_alpha * c / delta_r : 0.0;
    for (int j = 0; j < nz; ++j)
        s->dB_c[j] = j < pb ? pml_profile_len(c, delta_b, delta_b - (s->zv[j] + 0.5 * s->dz[j]), s->g.pml_R) : 0.0;
    for (int j = 0; j <= nz; ++j)
        s->dB_v[j] = j < pb ? pml_profile_len(c, delta_b, delta_b - s->zv[j], s->g.pml_R) : 0.0;
    for (int i = 0; i < nr; ++i)
        s->dR_c[i] = i >= nr - pr ? pml_profile_len(c, delta_r, s->rc[i] - r_in, s->g.pml_R) : 0.0;
    for (int i = 0; i <= nr; ++i)
        s->dR_v[i] = i > nr - pr ? pml_profile_len(c, delta_r, s->rR[i] - r_in, s->g.pml_R) : 0.0;
    /* the right strip absorbs waves of the medium: it acts on the rows whose reference
       (far-field) state holds material, not on the void above the target, where the
       reference is empty and damping toward it would remove ejecta (reading of Sect. 3) */
    for (int j = 0; j < nz; ++j) s->wR_c[j] = s->rho_ref[j] > 0.0 ? 1.0 : 0.0;
    for (int j = 0; j <= nz; ++j)
        s->wR_v[j] = ((j > 0 && s->rho_ref[j - 1] > 0.0) || (j < nz && s->rho_ref[j] > 0.0)) ? 1.0 : 0.0;
    s->finalized = 1;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Phase 0: EoS, artificial viscosity and the Courant time step.
 *   p_hat = sum_m f_m max(p_m, (1-D) p_t,m w_m)   (void carries no pressure; w_m the
 *   expansion weight)
 *   q = rho_bar (c_Q L^2 div^2 - c_L L c div) when div v < 0            (Amsden 1980)
 *   P = p_hat + Phi q,   Phi = sum_m f_m
 *   dt = min(C0 min_cells L / (max_vertex |v| + c), growth dt_prev, dt_max)   (Eq. 14)
 * L = min(dr, dz) of the cell (the cell size dx on a uniform grid).
 * Pinned by test_oracle_sod.py (shock capturing) and test_oracle_dt.py (hand-computed
 * dt on a 2x2 grid).
 * ------------------------------------------------------------------------------------ */
static double cell_div(const orc_sim* s, const double* vr, const double* vz, int i, int j)
{
    double uL = 0.5 * (vr[VID(s, i, j)] + vr[VID(s, i, j + 1)]);
    double uR = 0.5 * (vr[VID(s, i + 1, j)] + vr[VID(s, i + 1, j + 1)]);
    double uB = 0.5 * (vz[VID(s, i, j)] + vz[VID(s, i + 1, j)]);
    double uT = 0.5 * (vz[VID(s, i, j + 1)] + vz[VID(s, i + 1, j + 1)]);
    double flux = face_r(s, i + 1, j) * uR - face_r(s, i, j) * uL + s->A_Z[i] * (uT - uB);
    return flux / vol(s, i, j);
}

static void phase0_eos_dt(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz;
    double cand_min = INFINITY;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            int c = CID(s, i, j);
            double phat, phi, c2, rb;
            cell_eos(s, c, &phat, &phi, &c2, &rb);
            if (!(phi > 0.0)) { s->P[c] = 0.0; s->pbar[c] = 0.0; continue; }
            double cs = sqrt(c2);
            double div = cell_div(s, s->vr, s->vz, i, j);
            double dx = cell_len(s, i, j);
            double q = 0.0;
            if (div < 0.0) q = rb * (s->g.av_cq * dx * dx * div * div - s->g.av_cl * dx * cs * div);
            s->P[c] = phat + phi * q;
            s->pbar[c] = phat / phi;
            double over = s->pbar[c] - s->p0[j];
            if (over > s->pmax[c]) s->pmax[c] = over;
            double w = 0.0;
            int vv[4] = {VID(s, i, j), VID(s, i + 1, j), VID(s, i + 1, j + 1), VID(s, i, j + 1)};
            for (int k = 0; k < 4; ++k) {
                double u2 = s->vr[vv[k]] * s->vr[vv[k]] + s->vz[vv[k]] * s->vz[vv[k]];
                if (!(u2 <= w)) w = u2;     /* the larger speed; a NaN speed is kept (failure) */
            }
            double cand = dx / (sqrt(w) + cs);
            if (cand != cand) s->status |= 2;
            if (cand < cand_min) cand_min = cand;
        }
    }
    double dt = s->g.dt_growth * s->dt_prev;
    if (s->g.cfl * cand_min < dt) dt = s->g.cfl * cand_min;
    if (s->g.dt_max < dt) dt = s->g.dt_max;
    if (dt < s->g.dt_min) s->status |= 4;
    s->dt = dt;
}

/* ------------------------------------------------------------------------------------
 * Deviatoric corner forces of one cell on its four vertices (a = (i,j), b = (i+1,j),
 * c = (i+1,j+1), d = (i,j+1)): the negative gradient of the cell's deviatoric stress power
 * V (S_rr e_rr + S_zz e_zz + S_tt e_tt + 2 S_rz e_rz) with respect to the vertex
 * velocities (Eq. 1 in weak form), with the hoop stress S_tt = -(S_rr + S_zz).  Each
 * force is split into the part from r-derivatives ("radial") and the part from
 * z-derivatives ("vertical"), which the PML stress auxiliary psi1 needs (Eqs. 16, 21).
 * out[k] = (F_r radial, F_z radial, F_r vertical, F_z vertical) for corner k.
 * The isotropic part -P (A_R uR - A_L uL + A_Z (uT - uB)) is applied per vertex in
 * pressure-difference form (phase 1), so a uniform pressure cancels exactly.
 * Pinned by test_oracle_rest.py, test_oracle_conservation.py and test_oracle_strength
 * (through the pure-shear driver of the same stress power).
 * ------------------------------------------------------------------------------------ */
static void corner_forces_dev(const orc_sim* s, int i, int j, double Srr, double Szz, double Srz, double out[4][4])
{
    double hoop = 0.25 * s->dr[i] * s->dz[j];   /* V / (4 r_c) */
    double Stt = -(Srr + Szz);
    double hr = 0.5 * s->rc[i] * s->dz[j];      /* V / (2 dr) */
    double hz = 0.5 * s->A_Z[i];                /* V / (2 dz) */
    /* radial part: V (S_rr e_rr + S_tt e_tt + S_rz dvz/dr) */
    out[0][0] = hr * Srr - hoop * Stt;   out[0][1] = hr * Srz;
    out[1][0] = -hr * Srr - hoop * Stt;  out[1][1] = -hr * Srz;
    out[2][0] = -hr * Srr - hoop * Stt;  out[2][1] = -hr * Srz;
    out[3][0] = hr * Srr - hoop * Stt;   out[3][1] = hr * Srz;
    /* vertical part: V (S_zz e_zz + S_rz dvr/dz) */
    out[0][2] = hz * Srz;   out[0][3] = hz * Szz;
    out[1][2] = hz * Srz;   out[1][3] = hz * Szz;
    out[2][2] = -hz * Srz;  out[2][3] = -hz * Szz;
    out[3][2] = -hz * Srz;  out[3][3] = -hz * Szz;
}

static double cell_mass(const orc_sim* s, int c, int i)
{
    double m = 0.0;
    for (int k = 0; k < s->g.nmat; ++k) m += s->f[k][c] * s->rho[k][c];
    return m * vol(s, i, c / s->g.nr);
}

static double cell_phi(const orc_sim* s, int c)
{
    double f = 0.0;
    for (int k = 0; k < s->g.nmat; ++k) f += s->f[k][c];
    return f;
}

static void apply_velocity_bc(const orc_sim* s, int i, int j, double* vr, double* vz)
{
    if (i == 0 || i == s->g.nr) *vr = 0.0;
    if (j == 0) {
        *vz = 0.0;
        if (s->g.bc_bottom == ORC_BOTTOM_NOSLIP) *vr = 0.0;
    }
    if (j == s->g.nz && s->g.bc_top == ORC_TOP_WALL) *vz = 0.0;
}

/* ------------------------------------------------------------------------------------
 * Phase 1: Lagrangian momentum, Eq. 1, on the vertices:
 *   m_v = 1/4 sum of the adjacent cell masses,
 *   psi1 <- psi1 - dt d F_tangential(P - Phi p0)          (Sect. 3, Eqs. 16 and 21)
 *   v^L = v + dt ((F - psi1_b - psi1_r) / m_v + g)
 * F_tangential is the r-derivative part in the bottom strip and the z-derivative part in
 * the right strip (the x-strip psi1 takes the y-derivative: the printed d_x d/dx is read
 * as d/dy, by symmetry with the other x-strip auxiliaries).
 * ------------------------------------------------------------------------------------ */
static void phase1_vertex(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz;
    double dt = s->dt;
    for (int j = 0; j <= nz; ++j) {
        for (int i = 0; i <= nr; ++i) {
            int v = VID(s, i, j);
            /* cells around the vertex: 0 = (i-1,j-1), 1 = (i,j-1), 2 = (i,j), 3 = (i-1,j);
               the vertex is corner c, d, a, b of them respectively */
            int ci_list[4] = {i - 1, i, i, i - 1};
            int cj_list[4] = {j - 1, j - 1, j, j};
            int corner[4] = {2, 3, 0, 1};
            double Pc[4] = {0, 0, 0, 0}, Pp[4] = {0, 0, 0, 0};
            double devr = 0.0, devz = 0.0, mass = 0.0;
            double Tr_b = 0.0, Tz_b = 0.0, Tr_r = 0.0, Tz_r = 0.0;
            const double dRv = s->dR_v[i] * s->wR_v[j];
            int pml = s->dB_v[j] > 0.0 || dRv > 0.0;
            for (int k = 0; k < 4; ++k) {
                int ci = ci_list[k], cj = cj_list[k];
                if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                int c = CID(s, ci, cj);
                double phi = cell_phi(s, c);
                double out[4][4];
                corner_forces_dev(s, ci, cj, phi * s->srr[c], phi * s->szz[c], phi * s->srz[c], out);
                int q = corner[k];
                devr += out[q][0] + out[q][2];
                devz += out[q][1] + out[q][3];
                if (pml) {
                    Tr_b += out[q][0]; Tz_b += out[q][1];
                    Tr_r += out[q][2]; Tz_r += out[q][3];
                }
                Pc[k] = s->P[c];
                Pp[k] = s->P[c] - phi * s->p0[cj];
                mass += 0.25 * cell_mass(s, c, ci);
            }
            /* isotropic forces in difference form: radial through the face r_i of rows j-1
               and j, vertical through the faces z_j of columns i-1 and i */
            double ARb = j > 0 ? face_r(s, i, j - 1) : 0.0, ARt = j < nz ? face_r(s, i, j) : 0.0;
            double AZl = i > 0 ? s->A_Z[i - 1] : 0.0, AZr = i < nr ? s->A_Z[i] : 0.0;
            double Fr = 0.5 * (ARb * (Pc[0] - Pc[1]) + ARt * (Pc[3] - Pc[2])) + devr;
            double Fz = 0.5 * (AZl * (Pc[0] - Pc[3]) + AZr * (Pc[1] - Pc[2])) + devz;
            if (pml) {
                Tr_b += 0.5 * (ARb * (Pp[0] - Pp[1]) + ARt * (Pp[3] - Pp[2]));
                Tz_r += 0.5 * (AZl * (Pp[0] - Pp[3]) + AZr * (Pp[1] - Pp[2]));
            }
            s->psi1r_b[v] = s->psi1r_b[v] * (1.0 - s->alpha_b * dt) - dt * s->dB_v[j] * Tr_b;
            s->psi1z_b[v] = s->psi1z_b[v] * (1.0 - s->alpha_b * dt) - dt * s->dB_v[j] * Tz_b;
            s->psi1r_r[v] = s->psi1r_r[v] * (1.0 - s->alpha_r * dt) - dt * dRv * Tr_r;
            s->psi1z_r[v] = s->psi1z_r[v] * (1.0 - s->alpha_r * dt) - dt * dRv * Tz_r;
            s->mv[v] = mass;
            double vr = 0.0, vz = 0.0;
            if (mass > 0.0) {
                double ar = (Fr - s->psi1r_b[v] - s->psi1r_r[v]) / mass;
                double az = (Fz - s->psi1z_b[v] - s->psi1z_r[v]) / mass - s->g.gravity;
                vr = s->vr[v] + dt * ar;
                vz = s->vz[v] + dt * az;
            }
            apply_velocity_bc(s, i, j, &vr, &vz);
            s->vLr[v] = vr;
            s->vLz[v] = vz;
            /* the cells did work F.v^L dt but the vertex gained F.v^L dt - m|dv|^2/2 of
               kinetic energy; the difference goes back to the cells as heat (phase 3c) */
            double dvr = vr - s->vr[v], dvz = vz - s->vz[v];
            s->dK[v] = 0.5 * mass * (dvr * dvr + dvz * dvz);
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Elasto-plastic stress update of one cell (Sect. 1: elasto-plastic constitutive model,
 * Collins et al. 2004 strength, fragmentation by a scalar damage):
 *   Jaumann predictor  s* = s + dt (2 G eps_dot' + W s - s W),  W_rz = omega
 *   von Mises return   s = s* Y / sqrt(J2*)  when J2* > Y^2
 *   damage             D += (sqrt(J2*) - Y) / (sqrt(3) G) * inv_epsf,  D <= 1
 * sv = (s_rr, s_zz, s_rz, D) in/out; rates = (e_rr, e_zz, e_tt, e_rz, omega).
 * With G = 0 (no strength) the deviator is zero and D is unchanged.
 * Pinned by test_oracle_strength.py (elastic slope 2G, yield plateau, equivalent plastic
 * strain of pure shear, objective rotation).
 * ------------------------------------------------------------------------------------ */
static void stress_update(double sv[4], const double rates[5], double G, double Y, double inv_epsf, double dt)
{
    double srr = sv[0], szz = sv[1], srz = sv[2], D = sv[3];
    double err = rates[0], ezz = rates[1], ett = rates[2], erz = rates[3], omega = rates[4];
    if (G > 0.0) {
        double tr3 = (err + ezz + ett) / 3.0;
        double nrr = srr + dt * (2.0 * G * (err - tr3) + 2.0 * omega * srz);
        double nzz = szz + dt * (2.0 * G * (ezz - tr3) - 2.0 * omega * srz);
        double nrz = srz + dt * (2.0 * G * erz + omega * (szz - srr));
        double ntt = -(nrr + nzz);
        double J2 = 0.5 * (nrr * nrr + nzz * nzz + ntt * ntt) + nrz * nrz;
        if (J2 > Y * Y) {
            double sq = sqrt(J2);
            double k = Y / sq;
            nrr *= k; nzz *= k; nrz *= k;
            double deps = (sq - Y) / (sqrt(3.0) * G);
            D += deps * inv_epsf;
            if (D > 1.0) D = 1.0;
        }
        srr = nrr; szz = nzz; srz = nrz;
    } else {
        srr = 0.0; szz = 0.0; srz = 0.0;
    }
    sv[0] = srr; sv[1] = szz; sv[2] = srz; sv[3] = D;
}

void orc_stress_update(double sv[4], const double rates[5], double G, double Y, double inv_epsf, double dt)
{
    stress_update(sv, rates, G, Y, inv_epsf, dt);
}

/* ------------------------------------------------------------------------------------
 * Phase 2: Lagrangian energy (Eq. 2), volume change, strength and damage per cell, all
 * from the Lagrangian velocities v^L:
 *   dV = dt (A_R uR - A_L uL + A_Z (uT - uB)),  V^L = V + dV
 *   E^L = E - P dV + dt V (S:eps_dot) - dt psi2,   psi2 <- psi2 - dt d Pi_tangential
 *   volume change: matter and void share dV in proportion to their fractions in
 *   compression and in expansion (equal strain: the material work sum_m -p_m dV_m is then
 *   the -P dV charged to the energy); materials share the matter part pro rata;
 *   Jaumann elastic predictor, von Mises return to Y(p, D), damage += eps_p / eps_f.
 * Pinned by test_oracle_strength.py (pure-shear driver), test_oracle_conservation.py and
 * test_oracle_rh.py.
 * ------------------------------------------------------------------------------------ */
static void phase2_cell(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz, nm = s->g.nmat;
    double dt = s->dt;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            int c = CID(s, i, j);
            int va = VID(s, i, j), vb = VID(s, i + 1, j), vc = VID(s, i + 1, j + 1), vd = VID(s, i, j + 1);
            double phi = cell_phi(s, c);
            double V = vol(s, i, j);
            double rc = s->rc[i];
            if (!(phi > 0.0)) {
                /* empty cell: nothing to update; remap sees zero material */
                s->VL[c] = V + dt * (face_r(s, i + 1, j) * 0.5 * (s->vLr[vb] + s->vLr[vc])
                                     - face_r(s, i, j) * 0.5 * (s->vLr[va] + s->vLr[vd])
                                     + s->A_Z[i] * (0.5 * (s->vLz[vd] + s->vLz[vc]) - 0.5 * (s->vLz[va] + s->vLz[vb])));
                for (int m = 0; m < nm; ++m) { s->fL[m][c] = 0.0; s->rhoL[m][c] = 0.0; }
                s->IL[c] = 0.0; s->srrL[c] = 0.0; s->szzL[c] = 0.0; s->srzL[c] = 0.0; s->DL[c] = 0.0;
                continue;
            }
            double uL = 0.5 * (s->vLr[va] + s->vLr[vd]);
            double uR = 0.5 * (s->vLr[vb] + s->vLr[vc]);
            double uB = 0.5 * (s->vLz[va] + s->vLz[vb]);
            double uT = 0.5 * (s->vLz[vd] + s->vLz[vc]);
            double err = (uR - uL) / s->dr[i];
            double ezz = (uT - uB) / s->dz[j];
            double ett = (uR + uL) / (2.0 * rc);
            double dvr_dz = 0.5 * ((s->vLr[vd] + s->vLr[vc]) - (s->vLr[va] + s->vLr[vb])) / s->dz[j];
            double dvz_dr = 0.5 * ((s->vLz[vb] + s->vLz[vc]) - (s->vLz[va] + s->vLz[vd])) / s->dr[i];
            double erz = 0.5 * (dvr_dz + dvz_dr);
            double omega = 0.5 * (dvr_dz - dvz_dr);
            double radial_flux = face_r(s, i + 1, j) * uR - face_r(s, i, j) * uL;
            double vertical_flux = s->A_Z[i] * (uT - uB);
            double dV = dt * (radial_flux + vertical_flux);
            double VL = V + dV;
            s->VL[c] = VL;
            /* energy */
            double P = s->P[c];
            double Srr = phi * s->srr[c], Szz = phi * s->szz[c], Srz = phi * s->srz[c];
            double Stt = -(Srr + Szz);
            double Pi_rad = -P * radial_flux + V * (Srr * err + Stt * ett + Srz * dvz_dr);
            double Pi_ver = -P * vertical_flux + V * (Szz * ezz + Srz * dvr_dz);
            s->psi2_b[c] = s->psi2_b[c] * (1.0 - s->alpha_b * dt) - dt * s->dB_c[j] * Pi_rad;
            s->psi2_r[c] = s->psi2_r[c] * (1.0 - s->alpha_r * dt) - dt * s->dR_c[i] * s->wR_c[j] * Pi_ver;
            double M = 0.0;
            for (int m = 0; m < nm; ++m) M += s->f[m][c] * s->rho[m][c] * V;
            double dE = -P * dV + dt * V * (Srr * err + Szz * ezz + Stt * ett + 2.0 * Srz * erz)
                        - dt * (s->psi2_b[c] + s->psi2_r[c]);
            s->IL[c] = M > 0.0 ? s->I[c] + dE / M : s->I[c];
            /* volume partition: matter and void share dV in proportion to their fractions */
            double dVmat = phi * dV;
            for (int m = 0; m < nm; ++m) {
                double fm = s->f[m][c];
                if (!(fm > 0.0)) { s->fL[m][c] = 0.0; s->rhoL[m][c] = 0.0; continue; }
                double Vm = fm * V;
                double VmL = Vm + (fm / phi) * dVmat;
                /* status: a present material with a non-positive Lagrangian volume or density */
                if (!(VmL > 0.0) || !(s->rho[m][c] > 0.0)) s->status |= 1;
                s->rhoL[m][c] = s->rho[m][c] * (Vm / VmL);
                s->fL[m][c] = VmL / VL;
            }
            /* strength and damage */
            double G = 0.0, Y = 0.0, inv_epsf = 0.0;
            for (int m = 0; m < nm; ++m) {
                double fm = s->f[m][c];
                if (!(fm > 0.0) || s->mat[m].strength != ORC_STR_COLLINS) continue;
                const orc_material* mm = &s->mat[m];
                G += fm * mm->G;
                Y += fm * collins_yield(mm, s->pbar[c], s->D[c], s->I[c], s->rho[m][c]);
                double ef = mm->B_dam * (s->pbar[c] - mm->p_bd);
                if (ef < mm->eps_fb) ef = mm->eps_fb;
                inv_epsf += fm / ef;
            }
            G /= phi; Y /= phi; inv_epsf /= phi;
            double sv[4] = {s->srr[c], s->szz[c], s->srz[c], s->D[c]};
            double rates[5] = {err, ezz, ett, erz, omega};
            stress_update(sv, rates, G, Y, inv_epsf, dt);
            s->srrL[c] = sv[0]; s->szzL[c] = sv[1]; s->srzL[c] = sv[2]; s->DL[c] = sv[3];
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Phase 3a: Eulerian donor-cell remap of the cells, Eqs. 3-5, plus the PML mass and
 * energy terms of the control equations (Eqs. 23, 25): phi1, phi3 take d times the
 * tangential flux divergence, then M <- M - dt (d (M - M_ref) + phi1), likewise E.
 * Swept volume of a face dV_f = dt A_f u_f(v^L); the donor is the upwind cell; material m
 * moves f_m^L |dV_f| of volume at rho_m^L, energy moves with mass, stress and damage move
 * with matter volume.  Inflow through the top boundary is void.
 * Pinned by test_oracle_conservation.py (mass, IE), test_oracle_sod.py, test_oracle_pml.py.
 * ------------------------------------------------------------------------------------ */
typedef struct { double V[ORC_MAXMAT], M[ORC_MAXMAT], E, Srr, Szz, Srz, D; } orc_flux;

static void face_flux(const orc_sim* s, int donor, double dVabs, orc_flux* fl)
{
    memset(fl, 0, sizeof(*fl));
    if (donor < 0) return;
    double vmat = 0.0, mass = 0.0;
    for (int m = 0; m < s->g.nmat; ++m) {
        double dv = dVabs * s->fL[m][donor];
        fl->V[m] = dv;
        fl->M[m] = s->rhoL[m][donor] * dv;
        vmat += dv;
        mass += fl->M[m];
    }
    fl->E = s->IL[donor] * mass;
    fl->Srr = s->srrL[donor] * vmat;
    fl->Szz = s->szzL[donor] * vmat;
    fl->Srz = s->srzL[donor] * vmat;
    fl->D = s->DL[donor] * vmat;
}

static void phase3_remap(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz, nm = s->g.nmat;
    double dt = s->dt;
    size_t nc = s->ncell;
    /* new conserved totals, start from the Lagrangian cell contents */
    double* Vm[ORC_MAXMAT]; double* Mm[ORC_MAXMAT];
    for (int m = 0; m < nm; ++m) { Vm[m] = zalloc(nc); Mm[m] = zalloc(nc); }
    double* E = zalloc(nc); double* SV[4]; for (int k = 0; k < 4; ++k) SV[k] = zalloc(nc);
    double* FR_M = zalloc(nc); double* FZ_M = zalloc(nc);   /* net radial / vertical mass outflow */
    double* FR_E = zalloc(nc); double* FZ_E = zalloc(nc);
    for (int j = 0; j < nz; ++j) for (int i = 0; i < nr; ++i) {
        int c = CID(s, i, j);
        double vmat = 0.0, mass = 0.0;
        for (int m = 0; m < nm; ++m) {
            double v = s->fL[m][c] * s->VL[c];
            Vm[m][c] = v;
            Mm[m][c] = s->rhoL[m][c] * v;
            vmat += v; mass += Mm[m][c];
        }
        E[c] = s->IL[c] * mass;
        SV[0][c] = s->srrL[c] * vmat; SV[1][c] = s->szzL[c] * vmat;
        SV[2][c] = s->srzL[c] * vmat; SV[3][c] = s->DL[c] * vmat;
    }
    /* radial faces r_i, rows j: i = 1..nr-1 interior; i = 0 axis and i = nr wall carry nothing */
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i <= nr; ++i) {
            int f = j * (nr + 1) + i;
            double u = 0.5 * (s->vLr[VID(s, i, j)] + s->vLr[VID(s, i, j + 1)]);
            double dV = dt * face_r(s, i, j) * u;
            if (i == 0 || i == nr) dV = 0.0;
            s->dVR[f] = dV;
            orc_flux fl;
            int left = CID(s, i - 1, j), right = CID(s, i, j);
            int donor = dV > 0.0 ? left : (dV < 0.0 ? right : -1);
            face_flux(s, donor, fabs(dV), &fl);
            double sg = dV > 0.0 ? 1.0 : -1.0;
            double mass = 0.0;
            for (int m = 0; m < nm; ++m) mass += fl.M[m];
            s->dMR[f] = sg * mass;
            if (donor < 0) { s->dMR[f] = 0.0; continue; }
            /* out of the donor, into the acceptor */
            int acc = dV > 0.0 ? right : left;
            for (int m = 0; m < nm; ++m) {
                Vm[m][donor] -= fl.V[m]; Mm[m][donor] -= fl.M[m];
                Vm[m][acc] += fl.V[m]; Mm[m][acc] += fl.M[m];
            }
            E[donor] -= fl.E; E[acc] += fl.E;
            SV[0][donor] -= fl.Srr; SV[0][acc] += fl.Srr;
            SV[1][donor] -= fl.Szz; SV[1][acc] += fl.Szz;
            SV[2][donor] -= fl.Srz; SV[2][acc] += fl.Srz;
            SV[3][donor] -= fl.D; SV[3][acc] += fl.D;
            /* net radial outflow: the face is the right face of 'left' and the left face of 'right' */
            FR_M[left] += sg * mass; FR_M[right] -= sg * mass;
            FR_E[left] += sg * fl.E; FR_E[right] -= sg * fl.E;
        }
    }
    /* vertical faces z_j, columns i: j = 0 bottom wall, j = nz top boundary */
    for (int j = 0; j <= nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            int f = j * nr + i;
            double u = 0.5 * (s->vLz[VID(s, i, j)] + s->vLz[VID(s, i + 1, j)]);
            double dV = dt * s->A_Z[i] * u;
            if (j == 0) dV = 0.0;
            if (j == nz && s->g.bc_top == ORC_TOP_WALL) dV = 0.0;
            s->dVZ[f] = dV;
            int below = j > 0 ? CID(s, i, j - 1) : -1;
            int above = j < nz ? CID(s, i, j) : -1;
            int donor = dV > 0.0 ? below : (dV < 0.0 ? above : -1);
            orc_flux fl;
            face_flux(s, donor, fabs(dV), &fl);
            double sg = dV > 0.0 ? 1.0 : -1.0;
            double mass = 0.0;
            for (int m = 0; m < nm; ++m) mass += fl.M[m];
            s->dMZ[f] = donor < 0 ? 0.0 : sg * mass;
            if (donor < 0) continue;
            int acc = dV > 0.0 ? above : below;
            for (int m = 0; m < nm; ++m) {
                Vm[m][donor] -= fl.V[m]; Mm[m][donor] -= fl.M[m];
                if (acc >= 0) { Vm[m][acc] += fl.V[m]; Mm[m][acc] += fl.M[m]; }
            }
            E[donor] -= fl.E; SV[0][donor] -= fl.Srr; SV[1][donor] -= fl.Szz;
            SV[2][donor] -= fl.Srz; SV[3][donor] -= fl.D;
            if (acc >= 0) {
                E[acc] += fl.E; SV[0][acc] += fl.Srr; SV[1][acc] += fl.Szz;
                SV[2][acc] += fl.Srz; SV[3][acc] += fl.D;
            } else {
                /* outflow through the top */
                s->mass_out += mass;
                s->ie_out += fl.E;
            }
            if (below >= 0) { FZ_M[below] += sg * mass; FZ_E[below] += sg * fl.E; }
            if (above >= 0) { FZ_M[above] -= sg * mass; FZ_E[above] -= sg * fl.E; }
        }
    }
    /* new cell state, clean-up and the PML mass / energy terms.  Intensive quantities are
       updated in increment form, q' = q^L + (net flux of q-content - q^L net carrier flux)
       / new carrier amount, which is exact when nothing flows. */
    for (int j = 0; j < nz; ++j) for (int i = 0; i < nr; ++i) {
        int c = CID(s, i, j);
        double V = vol(s, i, j);
        double VmL[ORC_MAXMAT], MmL[ORC_MAXMAT], rho_new[ORC_MAXMAT];
        double MLtot = 0.0, VLmat = 0.0, dMtot = 0.0, dVtot = 0.0;
        for (int m = 0; m < nm; ++m) {
            VmL[m] = s->fL[m][c] * s->VL[c];
            MmL[m] = s->rhoL[m][c] * VmL[m];
            MLtot += MmL[m]; VLmat += VmL[m];
            /* Vm, Mm hold the Lagrangian contents plus the net fluxes */
            double dVm = Vm[m][c] - VmL[m], dMm = Mm[m][c] - MmL[m];
            dMtot += dMm; dVtot += dVm;
            rho_new[m] = Vm[m][c] > 0.0 ? s->rhoL[m][c] + (dMm - s->rhoL[m][c] * dVm) / Vm[m][c] : 0.0;
        }
        double Mtot = MLtot + dMtot, Vmat = VLmat + dVtot;
        double dE = E[c] - s->IL[c] * MLtot;
        double I = Mtot > 0.0 ? s->IL[c] + (dE - s->IL[c] * dMtot) / Mtot : 0.0;
        double srr = 0.0, szz = 0.0, srz = 0.0, D = 0.0;
        if (Vmat > 0.0) {
            srr = s->srrL[c] + ((SV[0][c] - s->srrL[c] * VLmat) - s->srrL[c] * dVtot) / Vmat;
            szz = s->szzL[c] + ((SV[1][c] - s->szzL[c] * VLmat) - s->szzL[c] * dVtot) / Vmat;
            srz = s->srzL[c] + ((SV[2][c] - s->srzL[c] * VLmat) - s->srzL[c] * dVtot) / Vmat;
            D = s->DL[c] + ((SV[3][c] - s->DL[c] * VLmat) - s->DL[c] * dVtot) / Vmat;
        }
        double Mkeep = 0.0, Vkeep = 0.0;
        for (int m = 0; m < nm; ++m) {
            double fm = Vm[m][c] / V;
            if (fm < s->g.f_min) {
                s->mass_discarded += Mm[m][c];
                Vm[m][c] = 0.0; Mm[m][c] = 0.0; rho_new[m] = 0.0;
            }
            Mkeep += Mm[m][c]; Vkeep += Vm[m][c];
        }
        if (!(Mkeep > 0.0)) { I = 0.0; srr = 0.0; szz = 0.0; srz = 0.0; D = 0.0; }
        /* PML auxiliaries take d times the tangential divergence: radial in the bottom
           strip, vertical in the right strip */
        s->phi1_b[c] = s->phi1_b[c] * (1.0 - s->alpha_b * dt) + s->dB_c[j] * FR_M[c];
        s->phi3_b[c] = s->phi3_b[c] * (1.0 - s->alpha_b * dt) + s->dB_c[j] * FR_E[c];
        const double dRc = s->dR_c[i] * s->wR_c[j];
        s->phi1_r[c] = s->phi1_r[c] * (1.0 - s->alpha_r * dt) + dRc * FZ_M[c];
        s->phi3_r[c] = s->phi3_r[c] * (1.0 - s->alpha_r * dt) + dRc * FZ_E[c];
        double dsum = s->dB_c[j] + dRc;
        double kappa = 1.0;
        if (Mkeep > 0.0 && dsum > 0.0) {
            double Mref = Vkeep * s->rho_ref[j];
            double dM = -dt * (dsum * (Mkeep - Mref) + s->phi1_b[c] + s->phi1_r[c]);
            double dEp = -dt * (dsum * (Mkeep * I - Mref * s->I_ref[j]) + s->phi3_b[c] + s->phi3_r[c]);
            double Mnew = Mkeep + dM;
            if (!(Mnew > 0.0)) s->status |= 1;
            s->mass_pml += dM;
            kappa = 1.0 + dM / Mkeep;
            I = I + (dEp - I * dM) / Mnew;
        }
        for (int m = 0; m < nm; ++m) {
            if (Vm[m][c] > 0.0) {
                s->f[m][c] = Vm[m][c] / V;
                s->rho[m][c] = kappa * rho_new[m];
            } else {
                s->f[m][c] = 0.0; s->rho[m][c] = 0.0;
            }
        }
        s->I[c] = I; s->srr[c] = srr; s->szz[c] = szz; s->srz[c] = srz; s->D[c] = D;
        if (I != I) s->status |= 2;
    }
    for (int m = 0; m < nm; ++m) { free(Vm[m]); free(Mm[m]); }
    free(E); for (int k = 0; k < 4; ++k) free(SV[k]);
    free(FR_M); free(FZ_M); free(FR_E); free(FZ_E);
}

/* ------------------------------------------------------------------------------------
 * Phase 3b: momentum remap on the dual (vertex) grid, Eq. 4.  The dual mass flux through
 * a dual face is the mean of the four cell-face mass fluxes it straddles (half of the two
 * boundary fluxes at the top boundary); momentum moves with the upwind vertex velocity;
 * the vertex mass is updated with the same fluxes.  PML: phi2 takes d times the
 * tangential dual momentum divergence, then P <- P - dt (d P + phi2) (Eq. 24).
 * Pinned by test_oracle_conservation.py (z-momentum; kinetic energy never grows in the
 * remap) and test_oracle_pml.py.
 * ------------------------------------------------------------------------------------ */
static double dMR_at(const orc_sim* s, int i, int j)   /* radial face r_i, row j */
{
    if (j < 0 || j >= s->g.nz) return 0.0;
    return s->dMR[j * (s->g.nr + 1) + i];
}
static double dMZ_at(const orc_sim* s, int i, int j)   /* vertical face z_j, column i */
{
    if (i < 0 || i >= s->g.nr) return 0.0;
    return s->dMZ[j * s->g.nr + i];
}

static double KRin(const orc_sim* s, const double* KR, const double* KZ, int i, int j)
{
    int nr = s->g.nr;
    double k = 0.0;
    if (i > 0) k += KR[j * nr + i - 1];
    if (j > 0) k += KZ[(j - 1) * (nr + 1) + i];
    return k;
}
static double KRout(const orc_sim* s, const double* KR, const double* KZ, int i, int j)
{
    int nr = s->g.nr;
    double k = KZ[j * (nr + 1) + i];
    if (i < nr) k += KR[j * nr + i];
    return k;
}

static void phase3_vertex(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz;
    double dt = s->dt;
    /* dual fluxes: radial dual face between (i,j) and (i+1,j): MR[j][i], i = 0..nr-1
       vertical dual face between (i,j) and (i,j+1): MZ[j][i], j = 0..nz-1; j = nz: top */
    double* MR = zalloc((size_t)(nz + 1) * nr);
    double* MZ = zalloc((size_t)(nz + 1) * (nr + 1));
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i < nr; ++i)
            MR[j * nr + i] = 0.25 * (dMR_at(s, i, j - 1) + dMR_at(s, i + 1, j - 1) + dMR_at(s, i, j) + dMR_at(s, i + 1, j));
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i <= nr; ++i)
            MZ[j * (nr + 1) + i] = 0.25 * (dMZ_at(s, i - 1, j) + dMZ_at(s, i - 1, j + 1) + dMZ_at(s, i, j) + dMZ_at(s, i, j + 1));
    for (int i = 0; i <= nr; ++i)
        MZ[nz * (nr + 1) + i] = 0.5 * (dMZ_at(s, i - 1, nz) + dMZ_at(s, i, nz));
    /* momentum fluxes with the upwind vertex velocity */
    double* PRr = zalloc((size_t)(nz + 1) * nr); double* PRz = zalloc((size_t)(nz + 1) * nr);
    double* PZr = zalloc((size_t)(nz + 1) * (nr + 1)); double* PZz = zalloc((size_t)(nz + 1) * (nr + 1));
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i < nr; ++i) {
            double m = MR[j * nr + i];
            int dv = m > 0.0 ? VID(s, i, j) : VID(s, i + 1, j);
            PRr[j * nr + i] = m * s->vLr[dv];
            PRz[j * nr + i] = m * s->vLz[dv];
        }
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i <= nr; ++i) {
            double m = MZ[j * (nr + 1) + i];
            int dv = (m > 0.0 || j == nz) ? VID(s, i, j) : VID(s, i, j + 1);
            PZr[j * (nr + 1) + i] = m * s->vLr[dv];
            PZz[j * (nr + 1) + i] = m * s->vLz[dv];
        }
    for (int i = 0; i <= nr; ++i) s->zmom_out += PZz[nz * (nr + 1) + i];
    /* kinetic energy fluxes 1/2 M |v_donor|^2 through the same dual faces */
    double* KR = zalloc((size_t)(nz + 1) * nr);
    double* KZ = zalloc((size_t)(nz + 1) * (nr + 1));
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i < nr; ++i) {
            double m = MR[j * nr + i];
            int dv = m > 0.0 ? VID(s, i, j) : VID(s, i + 1, j);
            KR[j * nr + i] = 0.5 * m * (s->vLr[dv] * s->vLr[dv] + s->vLz[dv] * s->vLz[dv]);
        }
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i <= nr; ++i) {
            double m = MZ[j * (nr + 1) + i];
            int dv = (m > 0.0 || j == nz) ? VID(s, i, j) : VID(s, i, j + 1);
            KZ[j * (nr + 1) + i] = 0.5 * m * (s->vLr[dv] * s->vLr[dv] + s->vLz[dv] * s->vLz[dv]);
        }
    for (int j = 0; j <= nz; ++j) {
        for (int i = 0; i <= nr; ++i) {
            int v = VID(s, i, j);
            double inR = i > 0 ? MR[j * nr + i - 1] : 0.0;
            double outR = i < nr ? MR[j * nr + i] : 0.0;
            double inZ = j > 0 ? MZ[(j - 1) * (nr + 1) + i] : 0.0;
            double outZ = MZ[j * (nr + 1) + i];
            double pinRr = i > 0 ? PRr[j * nr + i - 1] : 0.0, pinRz = i > 0 ? PRz[j * nr + i - 1] : 0.0;
            double poutRr = i < nr ? PRr[j * nr + i] : 0.0, poutRz = i < nr ? PRz[j * nr + i] : 0.0;
            double pinZr = j > 0 ? PZr[(j - 1) * (nr + 1) + i] : 0.0, pinZz = j > 0 ? PZz[(j - 1) * (nr + 1) + i] : 0.0;
            double poutZr = PZr[j * (nr + 1) + i], poutZz = PZz[j * (nr + 1) + i];
            double m = s->mv[v] + inR - outR + inZ - outZ;
            double pr = s->mv[v] * s->vLr[v] + pinRr - poutRr + pinZr - poutZr;
            double pz = s->mv[v] * s->vLz[v] + pinRz - poutRz + pinZz - poutZz;
            /* kinetic energy carried with the same upwind fluxes, minus what the remapped
               momentum holds: the donor-cell deficit, returned as heat */
            double kin = 0.5 * s->mv[v] * (s->vLr[v] * s->vLr[v] + s->vLz[v] * s->vLz[v])
                         + KRin(s, KR, KZ, i, j) - KRout(s, KR, KZ, i, j);
            double dKr = m > 0.0 ? kin - 0.5 * (pr * pr + pz * pz) / m : 0.0;
            s->kheat[v] = m > 0.0 ? (s->dK[v] + dKr) / m : 0.0;
            s->phi2r_b[v] = s->phi2r_b[v] * (1.0 - s->alpha_b * dt) + s->dB_v[j] * (poutRr - pinRr);
            s->phi2z_b[v] = s->phi2z_b[v] * (1.0 - s->alpha_b * dt) + s->dB_v[j] * (poutRz - pinRz);
            const double dRv = s->dR_v[i] * s->wR_v[j];
            s->phi2r_r[v] = s->phi2r_r[v] * (1.0 - s->alpha_r * dt) + dRv * (poutZr - pinZr);
            s->phi2z_r[v] = s->phi2z_r[v] * (1.0 - s->alpha_r * dt) + dRv * (poutZz - pinZz);
            double dsum = s->dB_v[j] + dRv;
            pr = pr - dt * (dsum * pr + s->phi2r_b[v] + s->phi2r_r[v]);
            pz = pz - dt * (dsum * pz + s->phi2z_b[v] + s->phi2z_r[v]);
            /* a vertex with no material in any adjacent cell after the clean-up carries
               no momentum (its dual mass is then only round-off of the fluxes) */
            int occupied = 0;
            for (int dj = -1; dj <= 0; ++dj) for (int di = -1; di <= 0; ++di) {
                int ci = i + di, cj = j + dj;
                if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                if (cell_phi(s, CID(s, ci, cj)) > 0.0) occupied = 1;
            }
            double vr = 0.0, vz = 0.0;
            if (m > 0.0 && occupied) { vr = pr / m; vz = pz / m; }
            apply_velocity_bc(s, i, j, &vr, &vz);
            s->vr[v] = vr;
            s->vz[v] = vz;
            if (vr != vr || vz != vz) s->status |= 2;
        }
    }
    free(MR); free(MZ); free(PRr); free(PRz); free(PZr); free(PZz); free(KR); free(KZ);
}

/* ------------------------------------------------------------------------------------
 * Phase 3c: the kinetic energy the step lost numerically at each vertex (the
 * symplectic-Euler deficit 1/2 m |dv|^2 and the donor-cell remap deficit) becomes
 * internal energy of the adjacent cells in proportion to their quarter masses:
 * I_c += 1/4 sum_{v in c} kheat_v with kheat_v = dK_v / m_v.  Total energy KE + IE is
 * then conserved to round-off without PML, outflow or clean-up.
 * Pinned by test_oracle_conservation.py and test_oracle_rh.py.
 * ------------------------------------------------------------------------------------ */
static void phase3_heat(orc_sim* s)
{
    int nr = s->g.nr, nz = s->g.nz;
    for (int j = 0; j < nz; ++j) for (int i = 0; i < nr; ++i) {
        int c = CID(s, i, j);
        double M = 0.0;
        for (int m = 0; m < s->g.nmat; ++m) M += s->f[m][c] * s->rho[m][c];
        if (!(M > 0.0)) continue;
        double add = 0.25 * (s->kheat[VID(s, i, j)] + s->kheat[VID(s, i + 1, j)]
                             + s->kheat[VID(s, i + 1, j + 1)] + s->kheat[VID(s, i, j + 1)]);
        s->I[c] += add;
    }
}

/* One full cycle (Fig. 1a): EoS and dt, Lagrangian step, Eulerian step. */
int orc_step(orc_sim* s, int nsteps)
{
    if (!s->finalized) return 1;
    for (int n = 0; n < nsteps; ++n) {
        phase0_eos_dt(s);
        phase1_vertex(s);
        phase2_cell(s);
        {
            double ke = 0.0, ie = 0.0;
            for (int v = 0; v < s->nvert; ++v) ke += 0.5 * s->mv[v] * (s->vLr[v] * s->vLr[v] + s->vLz[v] * s->vLz[v]);
            for (int j = 0; j < s->g.nz; ++j) for (int i = 0; i < s->g.nr; ++i) {
                int c = CID(s, i, j);
                double M = 0.0;
                for (int m = 0; m < s->g.nmat; ++m) M += s->f[m][c] * s->rho[m][c] * vol(s, i, j);
                ie += M * s->IL[c];
            }
            s->ke_lag = ke; s->ie_lag = ie;
        }
        phase3_remap(s);
        phase3_vertex(s);
        phase3_heat(s);
        s->t += s->dt;
        s->dt_prev = s->dt;
        s->nstep += 1;
    }
    return s->status;
}

/* Phase 0 alone on the current state (EoS, artificial viscosity, peak over-pressure and the
 * Courant step), without advancing: the total isotropic pressure P = p_hat + Phi q it forms
 * is then readable as field F_PTOTAL.  For the artificial-viscosity pins. */
int orc_phase0(orc_sim* s)
{
    if (!s->finalized) return 1;
    phase0_eos_dt(s);
    return s->status;
}

/* ------------------------------------------------------------------------------------
 * Field access.  Cell fields are row-major [j][i] (j = 0 at the bottom), vertex fields
 * [j][i] over (nr+1) x (nz+1).
 * ------------------------------------------------------------------------------------ */
enum {
    F_VOLFRAC0 = 0, F_VOLFRAC1 = 1, F_VOLFRAC2 = 2, F_DENS0 = 3, F_DENS1 = 4, F_DENS2 = 5,
    F_IE = 6, F_SRR = 7, F_SZZ = 8, F_SRZ = 9, F_DAMAGE = 10, F_PMAX = 11,
    F_VR = 12, F_VZ = 13, F_PRESSURE = 14, F_PTOTAL = 15,
    F_PHI1_B = 20, F_PHI3_B = 21, F_PSI2_B = 22, F_PHI1_R = 23, F_PHI3_R = 24, F_PSI2_R = 25,
    F_PHI2R_B = 30, F_PHI2Z_B = 31, F_PSI1R_B = 32, F_PSI1Z_B = 33,
    F_PHI2R_R = 34, F_PHI2Z_R = 35, F_PSI1R_R = 36, F_PSI1Z_R = 37
};

static double* field_ptr(orc_sim* s, int field, int* is_vertex)
{
    *is_vertex = 0;
    if (field >= F_VOLFRAC0 && field <= F_VOLFRAC2) return field - F_VOLFRAC0 < s->g.nmat ? s->f[field - F_VOLFRAC0] : NULL;
    if (field >= F_DENS0 && field <= F_DENS2) return field - F_DENS0 < s->g.nmat ? s->rho[field - F_DENS0] : NULL;
    switch (field) {
    case F_IE: return s->I; case F_SRR: return s->srr; case F_SZZ: return s->szz;
    case F_SRZ: return s->srz; case F_DAMAGE: return s->D; case F_PMAX: return s->pmax;
    case F_PTOTAL: return s->P;
    case F_PHI1_B: return s->phi1_b; case F_PHI3_B: return s->phi3_b; case F_PSI2_B: return s->psi2_b;
    case F_PHI1_R: return s->phi1_r; case F_PHI3_R: return s->phi3_r; case F_PSI2_R: return s->psi2_r;
    default: break;
    }
    *is_vertex = 1;
    switch (field) {
    case F_VR: return s->vr; case F_VZ: return s->vz;
    case F_PHI2R_B: return s->phi2r_b; case F_PHI2Z_B: return s->phi2z_b;
    case F_PSI1R_B: return s->psi1r_b; case F_PSI1Z_B: return s->psi1z_b;
    case F_PHI2R_R: return s->phi2r_r; case F_PHI2Z_R: return s->phi2z_r;
    case F_PSI1R_R: return s->psi1r_r; case F_PSI1Z_R: return s->psi1z_r;
    default: break;
    }
    return NULL;
}

int orc_get_field(orc_sim* s, int field, double* out, long n)
{
    if (field == F_PRESSURE) {
        if (n != s->ncell) return 1;
        for (int c = 0; c < s->ncell; ++c) {
            double phat, phi, c2, rb;
            cell_eos(s, c, &phat, &phi, &c2, &rb);
            out[c] = phi > 0.0 ? phat / phi : 0.0;
        }
        return 0;
    }
    int isv;
    double* p = field_ptr(s, field, &isv);
    if (!p) return 1;
    if (n != (isv ? s->nvert : s->ncell)) return 1;
    memcpy(out, p, sizeof(double) * (size_t)n);
    return 0;
}

int orc_set_field(orc_sim* s, int field, const double* in, long n)
{
    int isv;
    double* p = field_ptr(s, field, &isv);
    if (!p || field == F_PRESSURE || field == F_PTOTAL) return 1;
    if (n != (isv ? s->nvert : s->ncell)) return 1;
    memcpy(p, in, sizeof(double) * (size_t)n);
    return 0;
}

/* scalars: t, dt (of the last step), step count, status, tallies */
void orc_scalars(const orc_sim* s, double out[10])
{
    out[0] = s->t; out[1] = s->dt; out[2] = (double)s->nstep; out[3] = (double)s->status;
    out[4] = s->mass_out; out[5] = s->mass_discarded; out[6] = s->mass_pml; out[7] = s->zmom_out;
    out[8] = s->ke_lag; out[9] = s->ie_lag;
}

void orc_set_time(orc_sim* s, double t, double dt_prev)
{
    s->t = t;
    s->dt_prev = dt_prev;
}

/* Conservation sums (per radian): mass, z-momentum, kinetic energy, internal energy. */
void orc_conservation(const orc_sim* s, double out[4])
{
    double mass = 0.0, pz = 0.0, ke = 0.0, ie = 0.0;
    for (int j = 0; j < s->g.nz; ++j) for (int i = 0; i < s->g.nr; ++i) {
        int c = CID(s, i, j);
        double M = cell_mass(s, c, i);
        mass += M; ie += M * s->I[c];
    }
    for (int j = 0; j <= s->g.nz; ++j) for (int i = 0; i <= s->g.nr; ++i) {
        double m = 0.0;
        for (int dj = -1; dj <= 0; ++dj) for (int di = -1; di <= 0; ++di) {
            int ci = i + di, cj = j + dj;
            if (ci < 0 || ci >= s->g.nr || cj < 0 || cj >= s->g.nz) continue;
            m += 0.25 * cell_mass(s, CID(s, ci, cj), ci);
        }
        int v = VID(s, i, j);
        pz += m * s->vz[v];
        ke += 0.5 * m * (s->vr[v] * s->vr[v] + s->vz[v] * s->vz[v]);
    }
    out[0] = mass; out[1] = pz; out[2] = ke; out[3] = ie;
}

/* Point evaluations exported for the EoS / strength / profile pins. */
void orc_eos(const orc_material* m, double rho, double I, double* p, double* c2) { material_eos(m, rho, I, p, c2); }
double orc_yield(const orc_material* m, double p, double D, double I, double rho) { return collins_yield(m, p, D, I, rho); }
double orc_pml_profile(double c, double width, double dx, double y, double R) { return pml_profile(c, width, dx, y, R); }

/* ------------------------------------------------------------------------------------
 * Crater profile: surface height of each column where sum_m f_m crosses 1/2, scanning
 * down from the top, interpolated linearly between cell centres.
 * Pinned by test_oracle_crater.py (synthetic paraboloid bowl).
 * ------------------------------------------------------------------------------------ */
void orc_surface_heights(const orc_sim* s, double* h)
{
    int nr = s->g.nr, nz = s->g.nz;
    for (int i = 0; i < nr; ++i) {
        h[i] = 0.0;
        for (int j = nz - 1; j >= 0; --j) {
            double phi = cell_phi(s, CID(s, i, j));
            if (phi >= 0.5) {
                double zc = s->zv[j] + 0.5 * s->dz[j];
                if (j == nz - 1) { h[i] = zc; break; }
                double up = cell_phi(s, CID(s, i, j + 1));
                double zup = s->zv[j + 1] + 0.5 * s->dz[j + 1];
                h[i] = zc + (phi - 0.5) / (phi - up) * (zup - zc);
                break;
            }
        }
    }
}
