/*
 * FP64 CPU oracle of the Enskog-Vlasov lattice Boltzmann step
 * (Karlin & Hosseini, "Practical Kinetic Models for Dense Fluids", arXiv 2508.00577).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or table with
 * the CUDA path.
 *
 * It is written to be read against the paper: one plain loop over the nodes per
 * stage, every quantity stored in its own FP64 field, the stages in the order
 * in which the paper defines them.  Build with -ffp-contract=off so that no
 * multiply-add is fused; the expressions below fix the rounding order.
 *
 * Lattice: D2Q9 (Q=9) or D3Q27 (Q=27), velocities c_ia in {-1,0,1}, population
 * index i = (cx+1) + 3(cy+1) + 9(cz+1).  Fields are SoA with x fastest: node
 * n = x + nx*(y + ny*z); populations [Q][N]; vectors [D][N].  Boundaries are
 * periodic.  D2Q9 is read as the c_z-marginal of D3Q27 (3-D thermodynamics,
 * E = 3/2 RT + u^2/2); a D2Q9 lattice with nz > 1 is a stack of independent
 * 2-D layers, because no D2Q9 velocity or stencil reaches across z.
 *
 * Time step dt = 1 (lattice units).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int Q;            /* 9 (D2Q9) or 27 (D3Q27) */
    int nx, ny, nz;
    int eos;          /* 0: van der Waals form of the Enskog pressure; 1: Carnahan-Starling contact value */
    double a;         /* Vlasov attraction, P_V = -a rho^2 */
    double b;         /* excluded volume */
    double R;         /* gas constant */
    double kappa;     /* capillarity coefficient */
    double tau;       /* BARE relaxation time tau */
    double lambda;    /* relaxation time of the shifted equilibrium */
    int thermal;      /* 1: f and g populations; 0: temperature frozen, g absent */
    int force_form;   /* 0: divergence (Korteweg stress) form; 1: literal grad(a rho^2) + kappa rho grad(lap rho) */
    int walls;        /* 1: the columns x = 0 and x = nx-1 are wall nodes (see "Walls" below) */
    double wall_u[2][3];  /* velocity of the wall at x = 0 and at x = nx-1 */
    double wall_RT;   /* wall temperature R T_w */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Lattice                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int Q, D;
    int c[27][3];
    double w[27];     /* w_i = prod_a Psi_ia(0, 1/3): the rest equilibrium at theta = 1/3 */
} lattice;

static void make_lattice(int Q, lattice *L)
{
    L->Q = Q;
    L->D = (Q == 9) ? 2 : 3;
    for (int i = 0; i < Q; ++i) {
        L->c[i][0] = i % 3 - 1;
        L->c[i][1] = (i / 3) % 3 - 1;
        L->c[i][2] = (Q == 27) ? i / 9 - 1 : 0;
        double w = 1.0;
        for (int a = 0; a < L->D; ++a)
            w = w * ((L->c[i][a] == 0) ? (2.0 / 3.0) : (1.0 / 6.0));
        L->w[i] = w;
    }
}

static long node_shift(const orc_params *p, long n, int dx, int dy, int dz)
{
    long nx = p->nx, ny = p->ny, nz = p->nz;
    long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    x = (x + dx + nx) % nx;
    y = (y + dy + ny) % ny;
    z = (z + dz + nz) % nz;
    return x + nx * (y + ny * z);
}

/* Walls (the thermal Couette set-up of the paper's validation: u and T prescribed at
 * x = 0 and x = L_x).  The paper does not state its wall scheme; the reading used here
 * is a diffusely reflecting wall on the wall nodes.  With p->walls set, the lattice
 * columns x = 0 and x = nx-1 are wall nodes.  A wall node
 *   - does not stream: its moments, which the fluid nodes' stencils read, are those of
 *     its own populations,
 *   - carries no force (F = 0), so its moments are exactly (rho_w, u_w, R T_w),
 *   - does not collide: it absorbs the populations that stream into it from the fluid
 *     (mass m per step) and its populations become the equilibria
 *     f^eq(rho_w, u_w, theta0(rho_w, R T_w)) and g^eq(rho_w, u_w, R T_w) (Eqs. feq, geq)
 *     with rho_w such that the mass they send back into the fluid equals m: the
 *     populations moving off a wall with u_x = 0 carry rho_w theta0 / 2 = P_E(rho_w) / 2,
 *     so P_E(rho_w, R T_w) = 2 m (mass is conserved; energy is exchanged with the wall).
 * Nothing crosses between the two walls through the periodic x boundary as long as
 * kappa = 0 (the stress of a wall node then needs no density gradient). */
static int is_wall(const orc_params *p, long n)
{
    if (!p->walls)
        return 0;
    long x = n % p->nx;
    return x == 0 || x == p->nx - 1;
}

/* ------------------------------------------------------------------------ */
/* Product-form functions, Eq. (phi)                                         */
/* ------------------------------------------------------------------------ */

/* Psi_ia(xi, zeta) = 1 - c^2 + 1/2 [ (3c^2 - 2) zeta + c xi ]  (Eq. phi) */
static double Psi(int c, double xi, double zeta)
{
    double c2 = (double)(c * c);
    return 1.0 - c2 + 0.5 * ((3.0 * c2 - 2.0) * zeta + (double)c * xi);
}

/* The same linear combination applied to a polynomial sequence (A0, A1, A2),
 * i.e. Psi with the symbols 1, xi, zeta replaced by A0, A1, A2.  This is what
 * Psi(O, O^2) does to a function of u (Eq. geq). */
static double Psi_poly(int c, double A0, double A1, double A2)
{
    double c2 = (double)(c * c);
    return (1.0 - c2) * A0 + 0.5 * ((3.0 * c2 - 2.0) * A2 + (double)c * A1);
}

/* ------------------------------------------------------------------------ */
/* Equation of state (Enskog pressure P_E), gauge P0 = P_E (Eq. P0E)          */
/* ------------------------------------------------------------------------ */

/* Compressibility Z = P_E / (rho R T) and the pseudo-adiabatic exponent
 * gamma0 of Eq. (gamma) for P0 = P_E = rho RT Z(rho):
 *   gamma0 = (dlnP0/dlnrho)_T + 2/3 (P_E/(rho RT)) (dlnP0/dlnT)_rho
 *          = 1 + rho Z'(rho)/Z + 2/3 Z.
 * vdW form (the paper's P_E = rho RT/(1 - b rho)): rho Z'/Z = b rho Z, gamma0 = 5/3 Z.
 * Carnahan-Starling contact value, eta = b rho / 4:
 *   Z = (1 + eta + eta^2 - eta^3)/(1 - eta)^3,
 *   eta Z'/Z = eta (4 + 4 eta - 2 eta^2) / ((1 - eta)(1 + eta + eta^2 - eta^3)). */
static void eos_Z_gamma(int eos, int thermal, double b, double rho, double *Z, double *gamma0)
{
    double dlnZ;                                   /* rho Z'(rho) / Z */
    if (eos == 0) {
        *Z = 1.0 / (1.0 - b * rho);
        dlnZ = b * rho * *Z;
    } else {
        double eta = b * rho / 4.0;
        double num = 1.0 + eta + eta * eta - eta * eta * eta;
        double om = 1.0 - eta;
        *Z = num / (om * om * om);
        dlnZ = eta * (4.0 + 4.0 * eta - 2.0 * eta * eta) / (om * num);
    }
    /* With the temperature frozen (thermal = 0) the temperature term of Eq. (gamma)
     * drops out: gamma0 = (dlnP0/dlnrho)_T. */
    *gamma0 = thermal ? 1.0 + dlnZ + (2.0 / 3.0) * *Z : 1.0 + dlnZ;
}

void orc_eos(int eos, int thermal, double b, double rho, double RT, double *P0, double *theta0, double *gamma0)
{
    double Z, g0;
    eos_Z_gamma(eos, thermal, b, rho, &Z, &g0);
    *theta0 = RT * Z;
    *P0 = rho * *theta0;
    *gamma0 = g0;
}

/* ------------------------------------------------------------------------ */
/* Equilibria at one node                                                    */
/* ------------------------------------------------------------------------ */

/* f^eq_i = rho prod_a Psi_ia(u_a, theta0 + u_a^2)    (Eq. feq) with P0/rho = theta0.
 * The same call with (u*, zeta*) gives f* of Eq. (f_star) when zeta is passed. */
static void prod_eq(const lattice *L, double rho, const double xi[3], const double zeta[3], double *out)
{
    for (int i = 0; i < L->Q; ++i) {
        double p = 1.0;
        for (int a = 0; a < L->D; ++a)
            p = p * Psi(L->c[i][a], xi[a], zeta[a]);
        out[i] = rho * p;
    }
}

void orc_feq(int Q, double rho, const double *u, double theta0, double *out)
{
    lattice L;
    make_lattice(Q, &L);
    double zeta[3] = {0, 0, 0}, uu[3] = {0, 0, 0};
    for (int a = 0; a < L.D; ++a) {
        uu[a] = u[a];
        zeta[a] = theta0 + u[a] * u[a];
    }
    prod_eq(&L, rho, uu, zeta, out);
}

/* g^eq_i = rho prod_a Psi_ia(O_a, O_a^2) E(u, RT),  O_a A = theta0 dA/du_a + u_a A   (Eq. geq).
 * theta0 does not depend on u, so the O_a commute and each acts on u_a alone.
 * With E = e + 1/2 sum_b u_b^2 and e = 3/2 RT:
 *   O^k_a 1            = P_k(u_a):  P0 = 1, P1 = u, P2 = theta0 + u^2
 *   O^k_a (u_a^2 / 2)  = S_k(u_a):  S0 = u^2/2, S1 = theta0 u + u^3/2,
 *                                   S2 = theta0^2 + 5/2 theta0 u^2 + u^4/2
 * so g^eq_i = rho [ e prod_a PsiP_ia + sum_b PsiS_ib prod_{a != b} PsiP_ia ]
 * with PsiP = Psi_poly(c, P0, P1, P2) and PsiS = Psi_poly(c, S0, S1, S2). */
static void geq_node(const lattice *L, double rho, const double u[3], double theta0, double RT, double *out)
{
    double e = 1.5 * RT;
    for (int i = 0; i < L->Q; ++i) {
        double PsiP[3], PsiS[3];
        for (int a = 0; a < L->D; ++a) {
            double v = u[a];
            double S0 = 0.5 * v * v;
            double S1 = theta0 * v + 0.5 * v * v * v;
            double S2 = theta0 * theta0 + 2.5 * theta0 * v * v + 0.5 * v * v * v * v;
            PsiP[a] = Psi_poly(L->c[i][a], 1.0, v, theta0 + v * v);
            PsiS[a] = Psi_poly(L->c[i][a], S0, S1, S2);
        }
        double pP = 1.0;
        for (int a = 0; a < L->D; ++a)
            pP = pP * PsiP[a];
        double sS = 0.0;
        for (int b = 0; b < L->D; ++b) {
            double t = PsiS[b];
            for (int a = 0; a < L->D; ++a)
                if (a != b)
                    t = t * PsiP[a];
            sS = sS + t;
        }
        out[i] = rho * (e * pP + sS);
    }
}

void orc_geq(int Q, double rho, const double *u, double theta0, double RT, double *out)
{
    lattice L;
    make_lattice(Q, &L);
    double uu[3] = {0, 0, 0};
    for (int a = 0; a < L.D; ++a)
        uu[a] = u[a];
    geq_node(&L, rho, uu, theta0, RT, out);
}

/* ------------------------------------------------------------------------ */
/* Finite-difference operators (the paper does not fix them)                  */
/* ------------------------------------------------------------------------ */

/* Isotropic gradient: d_a phi = (1/cs^2) sum_i w_i c_ia phi(x + c_i), cs^2 = 1/3. */
static double grad_iso(const orc_params *p, const lattice *L, const double *phi, long n, int a)
{
    double acc = 0.0;
    for (int i = 0; i < L->Q; ++i)
        acc = acc + (L->w[i] * (double)L->c[i][a]) * phi[node_shift(p, n, L->c[i][0], L->c[i][1], L->c[i][2])];
    return 3.0 * acc;
}

/* Isotropic Laplacian: lap phi = (2/cs^2) sum_i w_i (phi(x + c_i) - phi(x)). */
static double lap_iso(const orc_params *p, const lattice *L, const double *phi, long n)
{
    double acc = 0.0;
    for (int i = 0; i < L->Q; ++i)
        acc = acc + L->w[i] * (phi[node_shift(p, n, L->c[i][0], L->c[i][1], L->c[i][2])] - phi[n]);
    return 6.0 * acc;
}

/* Central difference along axis a: (phi(x + e_a) - phi(x - e_a)) / 2. */
static double diff_c(const orc_params *p, const double *phi, long n, int a)
{
    int e[3] = {0, 0, 0};
    e[a] = 1;
    long np = node_shift(p, n, e[0], e[1], e[2]);
    long nm = node_shift(p, n, -e[0], -e[1], -e[2]);
    return 0.5 * (phi[np] - phi[nm]);
}

/* ------------------------------------------------------------------------ */
/* Work space                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    long N;
    double *fs, *gs;               /* streamed populations */
    double *rho, *j, *Gam;         /* raw moments */
    double *Pi, *lap, *A;          /* force intermediates */
    double *F, *u, *RT, *theta0, *P0, *gamma0, *flux, *wq;
    double *m_in;                  /* mass streaming into each wall node this step */
} work;

static int work_alloc(const orc_params *p, work *W)
{
    long N = (long)p->nx * p->ny * p->nz;
    int Q = p->Q;
    W->N = N;
    W->fs = malloc(sizeof(double) * Q * N);
    W->gs = malloc(sizeof(double) * Q * N);
    W->rho = malloc(sizeof(double) * N);
    W->j = malloc(sizeof(double) * 3 * N);
    W->Gam = malloc(sizeof(double) * N);
    W->Pi = malloc(sizeof(double) * 9 * N);
    W->lap = malloc(sizeof(double) * N);
    W->A = malloc(sizeof(double) * N);
    W->F = malloc(sizeof(double) * 3 * N);
    W->u = malloc(sizeof(double) * 3 * N);
    W->RT = malloc(sizeof(double) * N);
    W->theta0 = malloc(sizeof(double) * N);
    W->P0 = malloc(sizeof(double) * N);
    W->gamma0 = malloc(sizeof(double) * N);
    W->flux = malloc(sizeof(double) * 3 * N);
    W->wq = malloc(sizeof(double) * N);
    W->m_in = malloc(sizeof(double) * N);
    if (!W->m_in ||!W->fs || !W->gs || !W->rho || !W->j || !W->Gam || !W->Pi || !W->lap || !W->A || !W->F ||
        !W->u || !W->RT || !W->theta0 || !W->P0 || !W->gamma0 || !W->flux || !W->wq)
        return -1;
    return 0;
}

static void work_free(work *W)
{
    free(W->fs); free(W->gs); free(W->rho); free(W->j); free(W->Gam); free(W->Pi);
    free(W->lap); free(W->A); free(W->F); free(W->u); free(W->RT); free(W->theta0);
    free(W->P0); free(W->gamma0); free(W->flux); free(W->wq); free(W->m_in);
}

/* ------------------------------------------------------------------------ */
/* Stage 3: force                                                            */
/* ------------------------------------------------------------------------ */

/* Non-local force from the density field W->rho into W->F. */
static void force_stage(const orc_params *p, const lattice *L, work *W)
{
    const long N = W->N;
    const int D = L->D;

    /* Non-local force in the Enskog gauge P0 = P_E (Eq. P0E): the excluded-volume
     *    part cancels in Eq. (EVforce1) and the compression work of Eq. (Ework) vanishes,
     *    so F = -rho grad V_V = grad(a rho^2) + kappa rho grad(lap rho),  Q~ = 0. */
    if (p->force_form == 0) {
        /* Divergence form F_a = -d_b Pi_ab with the Korteweg stress
         * Pi_ab = (-a rho^2 - kappa rho lap rho - 1/2 kappa |grad rho|^2) delta_ab + kappa d_a rho d_b rho. */
#pragma omp parallel for schedule(static) if (N >= 4096)
        for (long n = 0; n < N; ++n) {
            double gr[3], rho = W->rho[n];
            for (int a = 0; a < D; ++a)
                gr[a] = grad_iso(p, L, W->rho, n, a);
            double lr = lap_iso(p, L, W->rho, n);
            double g2 = 0.0;
            for (int a = 0; a < D; ++a)
                g2 = g2 + gr[a] * gr[a];
            double s = -p->a * rho * rho - p->kappa * rho * lr - 0.5 * p->kappa * g2;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) {
                    double t = p->kappa * gr[a] * gr[b];
                    W->Pi[(a * 3 + b) * N + n] = (a == b) ? s + t : t;
                }
        }
#pragma omp parallel for schedule(static) if (N >= 4096)
        for (long n = 0; n < N; ++n)
            for (int a = 0; a < D; ++a) {
                double div = 0.0;
                for (int b = 0; b < D; ++b)
                    div = div + grad_iso(p, L, W->Pi + (a * 3 + b) * N, n, b);
                W->F[a * N + n] = -div;
            }
    } else {
        /* Literal form F = grad(a rho^2) + kappa rho grad(lap rho). */
#pragma omp parallel for schedule(static) if (N >= 4096)
        for (long n = 0; n < N; ++n) {
            W->lap[n] = lap_iso(p, L, W->rho, n);
            W->A[n] = p->a * W->rho[n] * W->rho[n];
        }
#pragma omp parallel for schedule(static) if (N >= 4096)
        for (long n = 0; n < N; ++n)
            for (int a = 0; a < D; ++a)
                W->F[a * N + n] = grad_iso(p, L, W->A, n, a) + p->kappa * W->rho[n] * grad_iso(p, L, W->lap, n, a);
    }
}

/* ------------------------------------------------------------------------ */
/* Stages 1-5: stream, moments, force, shifted velocity/energy, EOS           */
/* ------------------------------------------------------------------------ */

/* Everything the collision needs, computed from the post-collision state
 * (f, g) of the previous step.  RT_iso is the frozen RT field when thermal=0. */
static void macro_stages(const orc_params *p, const lattice *L, const double *f, const double *g,
                         const double *RT_iso, work *W)
{
    const long N = W->N;
    const int Q = L->Q, D = L->D;

    /* 1. Pull streaming: f_i(x) = f~_i(x - c_i)  (Eq. pre_LBM, exact on-lattice propagation).
     *    Wall nodes keep their own populations (walls, below). */
#pragma omp parallel for schedule(static) if (N >= 4096)
    for (long n = 0; n < N; ++n) {
        for (int i = 0; i < Q; ++i) {
            long src = is_wall(p, n) ? n : node_shift(p, n, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
            W->fs[i * N + n] = f[i * N + src];
            if (p->thermal)
                W->gs[i * N + n] = g[i * N + src];
        }
    }

    /* Walls: the mass streaming into each wall node, sum over the populations moving
     * toward it (c_x = -1 at x = 0, c_x = +1 at x = nx-1) pulled from the fluid. */
    if (p->walls)
        for (long n = 0; n < N; ++n) {
            W->m_in[n] = 0.0;
            if (!is_wall(p, n))
                continue;
            const int s = (n % p->nx) == 0 ? -1 : 1;
            for (int i = 0; i < Q; ++i)
                if (L->c[i][0] == s)
                    W->m_in[n] = W->m_in[n] + f[i * N + node_shift(p, n, -L->c[i][0], -L->c[i][1], -L->c[i][2])];
        }

    /* 2. Raw moments rho = sum f_i, j_a = sum c_ia f_i, Gamma = sum g_i  (ascending i). */
#pragma omp parallel for schedule(static) if (N >= 4096)
    for (long n = 0; n < N; ++n) {
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, Gam = 0.0;
        for (int i = 0; i < Q; ++i) {
            double fi = W->fs[i * N + n];
            rho = rho + fi;
            for (int a = 0; a < D; ++a)
                j[a] = j[a] + (double)L->c[i][a] * fi;
            if (p->thermal)
                Gam = Gam + W->gs[i * N + n];
        }
        W->rho[n] = rho;
        for (int a = 0; a < D; ++a)
            W->j[a * N + n] = j[a];
        W->Gam[n] = Gam;
    }

    /* 3. Non-local force in the Enskog gauge (stage above); none acts on wall nodes. */
    force_stage(p, L, W);
    if (p->walls)
        for (long n = 0; n < N; ++n)
            if (is_wall(p, n))
                for (int a = 0; a < D; ++a)
                    W->F[a * N + n] = 0.0;

    /* 4.-5. Shifted velocity (Eq. u_shift), energy (double-population analogue of
     *       Eq. T_shift with Q~ = 0), temperature, EOS and the corrected fluxes. */
#pragma omp parallel for schedule(static) if (N >= 4096)
    for (long n = 0; n < N; ++n) {
        double rho = W->rho[n], u[3] = {0, 0, 0}, F[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            F[a] = W->F[a * N + n];
            u[a] = (W->j[a * N + n] + 0.5 * F[a]) / rho;
        }
        double RT;
        if (p->thermal) {
            double uF = 0.0, u2 = 0.0;
            for (int a = 0; a < D; ++a) {
                uF = uF + u[a] * F[a];
                u2 = u2 + u[a] * u[a];
            }
            double E = (W->Gam[n] + 0.5 * uF) / rho;     /* rho E = Gamma + dt/2 (u.F + Q~) */
            RT = (2.0 / 3.0) * (E - 0.5 * u2);           /* rho E = 3/2 rho RT + 1/2 rho u^2 */
        } else {
            RT = RT_iso[n];
        }
        double P0, theta0, gamma0;
        orc_eos(p->eos, p->thermal, p->b, rho, RT, &P0, &theta0, &gamma0);
        W->RT[n] = RT;
        W->theta0[n] = theta0;
        W->P0[n] = P0;
        W->gamma0[n] = gamma0;
        for (int a = 0; a < D; ++a) {
            W->u[a * N + n] = u[a];
            /* rho u_a (u_a^2 + 3 P0/rho - 3 cs^2), cs^2 = 1/3   (Eq. correction_u) */
            W->flux[a * N + n] = rho * u[a] * (u[a] * u[a] + 3.0 * theta0 - 1.0);
        }
        W->wq[n] = theta0 - RT;                          /* P0/rho - RT   (Eq. correction_q) */
    }
}

/* ------------------------------------------------------------------------ */
/* Stages 6-8: gradient corrections, equilibria, collision                    */
/* ------------------------------------------------------------------------ */

static void collide_stage(const orc_params *p, const lattice *L, work *W, double *f, double *g)
{
    const long N = W->N;
    const int Q = L->Q, D = L->D;
    const double lambda = p->lambda;
    const double beta = 1.0 / (2.0 * p->tau + 1.0);          /* Eq. (beta), dt = 1 */
    const double c_eq = 2.0 * beta;
    const double c_star = (1.0 / lambda) * (1.0 - beta);       /* (dt/lambda)(1 - beta) */

#pragma omp parallel for schedule(static) if (N >= 4096)
    for (long n = 0; n < N; ++n) {
        if (is_wall(p, n))
            continue;
        double rho = W->rho[n], RT = W->RT[n], theta0 = W->theta0[n], P0 = W->P0[n];
        double u[3] = {0, 0, 0}, F[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            u[a] = W->u[a * N + n];
            F[a] = W->F[a * N + n];
        }

        /* 6. Gradient corrections, Eqs. (correction_u), (correction_gamma), (correction_q). */
        double divu = 0.0;
        for (int a = 0; a < D; ++a)
            divu = divu + diff_c(p, W->u + a * N, n, a);
        double Phi1 = P0 * (5.0 / 3.0 - W->gamma0[n]) * divu;
        /* Phi_aa = -d_a[rho u_a (u_a^2 + 3 P0/rho - 3 cs^2)] + Phi'.  The first term
         * cancels the lattice bias c_ia^3 = c_ia of the third moment; with the sign of
         * Eq. (correction_u) as printed it would double it (the Chapman-Enskog expansion
         * of Eq. (pre_LBM) needs the source (1 - beta)(Q_lattice - Q_Maxwell) in the
         * diagonal stress), which the adiabatic sound-attenuation test detects. */
        double Phi[3] = {0, 0, 0}, q[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            Phi[a] = Phi1 - diff_c(p, W->flux + a * N, n, a);
            q[a] = lambda * P0 * diff_c(p, W->wq, n, a) + lambda * u[a] * Phi1;
        }

        /* 7. Equilibria. f^eq (Eq. feq); f* with u* = u + lambda F/rho (Eq. def_ustar) and
         *    zeta* = P0/rho + u*^2 + lambda Phi/rho (Eq. f_star). */
        double us[3] = {0, 0, 0}, zeq[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            us[a] = u[a] + lambda * F[a] / rho;
            zeq[a] = theta0 + u[a] * u[a];
            zs[a] = theta0 + us[a] * us[a] + lambda * Phi[a] / rho;
        }
        double feq[27], fst[27];
        prod_eq(L, rho, u, zeq, feq);
        prod_eq(L, rho, us, zs, fst);

        /* 8. Collision h~ = h + 2 beta (h^eq - h) + (dt/lambda)(1 - beta)(h* - h^eq)  (Eq. pre_LBM). */
        for (int i = 0; i < Q; ++i) {
            double h = W->fs[i * N + n];
            f[i * N + n] = h + c_eq * (feq[i] - h) + c_star * (fst[i] - feq[i]);
        }

        if (p->thermal) {
            /* g^eq (Eq. geq) at (u, RT); g* = g^eq(u*, RT*) + g' (Eq. gstar) with
             * RT* = RT + 2 lambda/(3 rho) Q~ - lambda^2/(3 rho^2) F.F, Q~ = 0 (Eq. def_ustar),
             * P0/rho kept at (rho, RT); g'_i = 1/2 c_i.q' on the |c_i|^2 = 1 links (Eq. g_corr). */
            double FF = 0.0;
            for (int a = 0; a < D; ++a)
                FF = FF + F[a] * F[a];
            double RTs = RT - lambda * lambda / (3.0 * rho * rho) * FF;
            double geq[27], gst[27];
            geq_node(L, rho, u, theta0, RT, geq);
            geq_node(L, rho, us, theta0, RTs, gst);
            for (int i = 0; i < Q; ++i) {
                int c2 = 0;
                double cq = 0.0;
                for (int a = 0; a < D; ++a) {
                    c2 += L->c[i][a] * L->c[i][a];
                    cq = cq + (double)L->c[i][a] * q[a];
                }
                if (c2 == 1)
                    gst[i] = gst[i] + 0.5 * cq;
            }
            for (int i = 0; i < Q; ++i) {
                double h = W->gs[i * N + n];
                g[i * N + n] = h + c_eq * (geq[i] - h) + c_star * (gst[i] - geq[i]);
            }
        }
    }
}

/* Density rho_w of a wall node at temperature RT with P_E(rho_w, RT) = P (P_E
 * increases with rho): van der Waals form in closed form, rho = P / (RT + b P);
 * Carnahan-Starling by sixteen Newton steps from the ideal-gas value P / RT, with
 * dP_E/drho = RT d(eta Z)/d eta = RT (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4)/(1 - eta)^4. */
static double wall_density(const orc_params *p, double P, double RT)
{
    if (p->eos == 0)
        return P / (RT + p->b * P);
    double rho = P / RT;
    for (int k = 0; k < 16; ++k) {
        double eta = p->b * rho / 4.0;
        double num = 1.0 + eta + eta * eta - eta * eta * eta;
        double om = 1.0 - eta;
        double Z = num / (om * om * om);
        double dn = 1.0 + 4.0 * eta + 4.0 * eta * eta - 4.0 * eta * eta * eta + eta * eta * eta * eta;
        rho = rho - (rho * RT * Z - P) / (RT * (dn / (om * om * om * om)));
    }
    return rho;
}

/* Wall nodes after the collision: equilibria at the wall velocity and temperature with
 * the density that returns the absorbed mass (reading stated at is_wall). */
static void wall_stage(const orc_params *p, const lattice *L, const work *W, double *f, double *g)
{
    const long N = W->N;
    const long nx = p->nx;
    for (long n = 0; n < N; ++n) {
        if (!is_wall(p, n))
            continue;
        const long x = n % nx;
        const int side = x == 0 ? 0 : 1;
        double rho = wall_density(p, 2.0 * W->m_in[n], p->wall_RT), u[3], zeta[3] = {0, 0, 0}, out[27];
        double P0, theta0, gamma0;
        orc_eos(p->eos, p->thermal, p->b, rho, p->wall_RT, &P0, &theta0, &gamma0);
        for (int a = 0; a < 3; ++a)
            u[a] = a < L->D ? p->wall_u[side][a] : 0.0;
        for (int a = 0; a < L->D; ++a)
            zeta[a] = theta0 + u[a] * u[a];
        prod_eq(L, rho, u, zeta, out);
        for (int i = 0; i < L->Q; ++i)
            f[i * N + n] = out[i];
        if (p->thermal) {
            geq_node(L, rho, u, theta0, p->wall_RT, out);
            for (int i = 0; i < L->Q; ++i)
                g[i * N + n] = out[i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Entry points                                                              */
/* ------------------------------------------------------------------------ */

static int check(const orc_params *p)
{
    if (!p || (p->Q != 9 && p->Q != 27) || p->nx < 1 || p->ny < 1 || p->nz < 1)
        return -1;
    if (!(p->tau > 0.0) || !(p->lambda > 0.0))
        return -1;
    if (p->walls && (p->nx < 3 || p->kappa != 0.0 || !(p->wall_RT > 0.0)))
        return -1;
    return 0;
}

/* Initial populations (state = "post-collision" populations, streamed at the first step):
 * f = f^eq(rho0, u0, theta0(rho0, RT0)), g = g^eq(rho0, u0, RT0), RT0 = R T0.
 * u is [D][N]; T is [N].  g may be NULL when thermal = 0. */
int orc_init(const orc_params *p, const double *rho, const double *u, const double *T, double *f, double *g)
{
    if (check(p))
        return -1;
    lattice L;
    make_lattice(p->Q, &L);
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static) if (N >= 4096)
    for (long n = 0; n < N; ++n) {
        double uu[3] = {0, 0, 0}, zeta[3] = {0, 0, 0}, out[27];
        double RT = p->R * T[n], P0, theta0, gamma0;
        orc_eos(p->eos, p->thermal, p->b, rho[n], RT, &P0, &theta0, &gamma0);
        for (int a = 0; a < L.D; ++a) {
            uu[a] = u[a * N + n];
            zeta[a] = theta0 + uu[a] * uu[a];
        }
        prod_eq(&L, rho[n], uu, zeta, out);
        for (int i = 0; i < L.Q; ++i)
            f[i * N + n] = out[i];
        if (p->thermal && g) {
            geq_node(&L, rho[n], uu, theta0, RT, out);
            for (int i = 0; i < L.Q; ++i)
                g[i * N + n] = out[i];
        }
    }
    return 0;
}

/* Advance the state (f, g) in place by nsteps.  T_iso ([N], temperature) is read
 * only when thermal = 0. */
int orc_step(const orc_params *p, int nsteps, double *f, double *g, const double *T_iso)
{
    if (check(p) || nsteps < 0)
        return -1;
    lattice L;
    make_lattice(p->Q, &L);
    work W;
    if (work_alloc(p, &W)) {
        work_free(&W);
        return -2;
    }
    if (!p->thermal)
        for (long n = 0; n < W.N; ++n)
            W.RT[n] = p->R * T_iso[n];
    double *RT_iso = p->thermal ? NULL : malloc(sizeof(double) * W.N);
    if (!p->thermal)
        memcpy(RT_iso, W.RT, sizeof(double) * W.N);
    for (int s = 0; s < nsteps; ++s) {
        macro_stages(p, &L, f, g, RT_iso, &W);
        collide_stage(p, &L, &W, f, g);
        if (p->walls)
            wall_stage(p, &L, &W, f, g);
    }
    free(RT_iso);
    work_free(&W);
    return 0;
}

/* Macroscopic fields of the current state, as the next step would see them:
 * rho [N], u [D][N] (shifted, Eq. u_shift), T [N], F [D][N] (any output may be NULL). */
int orc_macro(const orc_params *p, const double *f, const double *g, const double *T_iso,
              double *rho, double *u, double *T, double *F)
{
    if (check(p))
        return -1;
    lattice L;
    make_lattice(p->Q, &L);
    work W;
    if (work_alloc(p, &W)) {
        work_free(&W);
        return -2;
    }
    double *RT_iso = NULL;
    if (!p->thermal) {
        RT_iso = malloc(sizeof(double) * W.N);
        for (long n = 0; n < W.N; ++n)
            RT_iso[n] = p->R * T_iso[n];
    }
    macro_stages(p, &L, f, g, RT_iso, &W);
    for (long n = 0; n < W.N; ++n) {
        if (rho) rho[n] = W.rho[n];
        if (T) T[n] = W.RT[n] / p->R;
        for (int a = 0; a < L.D; ++a) {
            if (u) u[a * W.N + n] = W.u[a * W.N + n];
            if (F) F[a * W.N + n] = W.F[a * W.N + n];
        }
    }
    free(RT_iso);
    work_free(&W);
    return 0;
}

/* Force of the Enskog gauge (stage 3 alone) for a given density field rho [N]:
 * F [D][N].  Used to check the stencils against analytic derivatives. */
int orc_force(const orc_params *p, const double *rho, double *F)
{
    if (check(p))
        return -1;
    lattice L;
    make_lattice(p->Q, &L);
    work W;
    if (work_alloc(p, &W)) {
        work_free(&W);
        return -2;
    }
    memcpy(W.rho, rho, sizeof(double) * W.N);
    force_stage(p, &L, &W);
    for (int a = 0; a < L.D; ++a)
        memcpy(F + a * W.N, W.F + a * W.N, sizeof(double) * W.N);
    work_free(&W);
    return 0;
}

/* Conserved totals of the state: out = { sum rho, sum j_x, sum j_y, sum j_z, sum g }
 * (raw population moments, summed over nodes in index order). */
int orc_totals(const orc_params *p, const double *f, const double *g, double *out)
{
    if (check(p))
        return -1;
    lattice L;
    make_lattice(p->Q, &L);
    const long N = (long)p->nx * p->ny * p->nz;
    for (int k = 0; k < 5; ++k)
        out[k] = 0.0;
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < L.Q; ++i) {
            double fi = f[i * N + n];
            out[0] += fi;
            for (int a = 0; a < 3; ++a)
                out[1 + a] += (double)L.c[i][a] * fi;
            if (p->thermal && g)
                out[4] += g[i * N + n];
        }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
