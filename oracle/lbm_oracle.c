/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the lattice Boltzmann-BGK (LBGK) method of
 * Colosqui, Karabacak, Ekinci & Yakhot, "Lattice Boltzmann simulation of high-frequency flows:
 * electromechanical resonators in gaseous media" (2009).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is compared against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library: every number below is typed from the
 * paper (or, for D2Q9, from the textbook lattice) and every step follows the paper's algorithm in
 * the paper's order, with full f (not deviations), array-of-structures storage and plain loops.
 *
 * Equation numbers follow the order of the numbered displays in the paper:
 *   Eq. 7  BE-BGK equation                      Eq. 12 bounce-back wall (BB)
 *   Eq. 8  Maxwellian equilibrium               Eq. 14 discrete LBGK equations
 *   Eq. 9  moments rho, rho u, energy            Eq. 15 second-order Hermite equilibrium (H2)
 *   Eq. 16 discrete moments                      Eq. 17 advection (streaming)
 *   Eq. 18 regularized BGK collision             Eq. 19 projected non-equilibrium part
 *   Appendix A, Table "D2Q37": velocity shells and weights.
 *
 * Readings where the paper is silent (each one also listed in the design notes):
 *   - lattice units dx = dt = 1 and lattice speed c = 1, so theta = 1/1.19697977039307^2;
 *   - the 4th-order equilibrium continues the Hermite (Taylor-in-u) series of Eq. 15;
 *   - node-return bounce-back on multi-speed links: a population whose pull source, or any lattice
 *     node strictly between source and destination, is solid comes back from the destination's own
 *     opposite population plus the moving-wall term of Eq. 12 (2 w_i rho0 c_i.U_w / theta);
 *   - the wall velocity and the body force of step n -> n+1 are evaluated at t = n + 1/2;
 *   - body force: Guo-type source with half-force velocity; in the regularized collision the
 *     projected non-equilibrium part keeps its first Hermite moment (zero without a force, -F/2
 *     with one), so that total momentum grows by exactly F per step;
 *   - force on the body: momentum exchange summed over every link blocked by a body node;
 *   - diffuse scattering (Eq. 11) on the lattice: at a fluid node, the populations coming back from
 *     a wall along its blocked links are the wall's discrete Maxwellian (the equilibrium of the
 *     run's order at the wall velocity) with the density that returns exactly the mass the node
 *     sends into that wall (zero net normal mass flux), per wall.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OQMAX 37

typedef struct {
    int Q;
    double theta;          /* c_s^2 in lattice units                                        */
    int c[OQMAX][2];       /* integer lattice velocities                                     */
    double w[OQMAX];       /* quadrature weights                                             */
    int opp[OQMAX];        /* index of -c_i                                                  */
} olat;

/* D2Q37 shells, Appendix A Table "D2Q37": one representative velocity (in units of the lattice
 * speed c) and its weight; all states of a shell follow from sign flips and the x<->y swap. */
static const int d2q37_shell_v[8][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 2}, {3, 0}, {1, 2}, {1, 3}};
static const double d2q37_shell_w[8] = {
    0.233150669132352000, 0.107306091542219000, 0.057667859888794800, 0.014208216158450700,
    0.001011937592673570, 0.000245301027757717, 0.005353049000513770, 0.000283414252994198};
static const int d2q37_shell_states[8] = {1, 4, 4, 4, 4, 4, 8, 8};

/* Textbook D2Q9 (not in the paper): rest 4/9, axis 1/9, diagonal 1/36, theta = 1/3. */
static const int d2q9_shell_v[3][2] = {{0, 0}, {1, 0}, {1, 1}};
static const double d2q9_shell_w[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
static const int d2q9_shell_states[3] = {1, 4, 4};

static int add_shell(olat* L, int vx, int vy, double w) {
    int start = L->Q, k, s;
    for (s = 0; s < 8; ++s) {
        int a = (s & 1) ? -vx : vx;
        int b = (s & 2) ? -vy : vy;
        int cx = (s & 4) ? b : a, cy = (s & 4) ? a : b, dup = 0;
        for (k = start; k < L->Q; ++k)
            if (L->c[k][0] == cx && L->c[k][1] == cy) dup = 1;
        if (!dup) {
            L->c[L->Q][0] = cx;
            L->c[L->Q][1] = cy;
            L->w[L->Q] = w;
            L->Q++;
        }
    }
    return L->Q - start;
}

static int build_lattice(int Q, olat* L) {
    int s, i, j;
    memset(L, 0, sizeof(*L));
    if (Q == 37) {
        for (s = 0; s < 8; ++s)
            if (add_shell(L, d2q37_shell_v[s][0], d2q37_shell_v[s][1], d2q37_shell_w[s]) != d2q37_shell_states[s])
                return -1;
        L->theta = 1.0 / (1.19697977039307 * 1.19697977039307);
    } else if (Q == 9) {
        for (s = 0; s < 3; ++s)
            if (add_shell(L, d2q9_shell_v[s][0], d2q9_shell_v[s][1], d2q9_shell_w[s]) != d2q9_shell_states[s])
                return -1;
        L->theta = 1.0 / 3.0;
    } else {
        return -1;
    }
    if (L->Q != Q) return -1;
    for (i = 0; i < Q; ++i) {
        L->opp[i] = -1;
        for (j = 0; j < Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1]) L->opp[i] = j;
        if (L->opp[i] < 0) return -1;
    }
    return 0;
}

/* Lattice tables for the test suite: c (Q x 2 ints), w (Q doubles), theta. */
int oracle_lattice(int Q, int* c, double* w, double* theta) {
    olat L;
    int i;
    if (build_lattice(Q, &L)) return -1;
    for (i = 0; i < Q; ++i) {
        c[2 * i] = L.c[i][0];
        c[2 * i + 1] = L.c[i][1];
        w[i] = L.w[i];
    }
    *theta = L.theta;
    return 0;
}

/* Eq. 15 (order 2): f_i^eq = w_i rho [1 + a + (a^2 - b)/2] with a = c_i.u/theta, b = u^2/theta.
 * Order 4 continues the same Hermite series of the Maxwellian (Eq. 8):
 *   + (a^3 - 3ab)/6 + (a^4 - 6a^2 b + 3b^2)/24. */
static void equilibrium(const olat* L, int order, double rho, double ux, double uy, double* feq) {
    int i;
    double b = (ux * ux + uy * uy) / L->theta;
    for (i = 0; i < L->Q; ++i) {
        double a = (L->c[i][0] * ux + L->c[i][1] * uy) / L->theta;
        double h = 1.0 + a + 0.5 * (a * a - b);
        if (order >= 4) h += (a * a * a - 3.0 * a * b) / 6.0 + (a * a * a * a - 6.0 * a * a * b + 3.0 * b * b) / 24.0;
        feq[i] = L->w[i] * rho * h;
    }
}

int oracle_equilibrium(int Q, int order, double rho, double ux, double uy, double* feq) {
    olat L;
    if (build_lattice(Q, &L) || (order != 2 && order != 4)) return -1;
    equilibrium(&L, order, rho, ux, uy, feq);
    return 0;
}

/* Eq. 19: projection of f^adv - f^eq onto the second-order Hermite space,
 *   fne_i = w_i/(2 theta^2) (c_ia c_ib - theta delta_ab) sum_j (f_j^adv - f_j^eq) c_ja c_jb,
 * plus the first-order part w_i c_i.J/theta with J = sum_j (f_j^adv - f_j^eq) c_j, which vanishes
 * when u = sum f c / rho (no body force) and equals -F/2 with the half-force velocity. */
static void project_nonequilibrium(const olat* L, const double* fadv, const double* feq, double* fne) {
    int i, j;
    double Jx = 0, Jy = 0, Pxx = 0, Pxy = 0, Pyy = 0, th = L->theta;
    for (j = 0; j < L->Q; ++j) {
        double d = fadv[j] - feq[j];
        Jx += d * L->c[j][0];
        Jy += d * L->c[j][1];
        Pxx += d * L->c[j][0] * L->c[j][0];
        Pxy += d * L->c[j][0] * L->c[j][1];
        Pyy += d * L->c[j][1] * L->c[j][1];
    }
    for (i = 0; i < L->Q; ++i) {
        double cx = L->c[i][0], cy = L->c[i][1];
        double second = (cx * cx - th) * Pxx + 2.0 * cx * cy * Pxy + (cy * cy - th) * Pyy;
        double first = cx * Jx + cy * Jy;
        fne[i] = L->w[i] * (first / th + second / (2.0 * th * th));
    }
}

int oracle_project(int Q, const double* fadv, const double* feq, double* fne) {
    olat L;
    if (build_lattice(Q, &L)) return -1;
    project_nonequilibrium(&L, fadv, feq, fne);
    return 0;
}

/* Guo-type body-force source (the paper moves the wall instead; the body-frame drive is a reading
 * of this build): with the fluid force density F = rho g and the half-force velocity u,
 *   S_i = (1 - 1/(2 tau)) w_i [ c_i.F/theta + ((c_i.u)(c_i.F) - theta u.F)/theta^2 ],
 * whose moments are 0, (1 - 1/(2 tau)) F and (1 - 1/(2 tau)) (uF + Fu). */
static void guo_source(const olat* L, double tau, double ux, double uy, double Fbx, double Fby, double* S) {
    int i;
    double th = L->theta;
    for (i = 0; i < L->Q; ++i) {
        double cx = L->c[i][0], cy = L->c[i][1];
        double cu = cx * ux + cy * uy, cF = cx * Fbx + cy * Fby, uF = ux * Fbx + uy * Fby;
        S[i] = (1.0 - 0.5 / tau) * L->w[i] * (cF / th + (cu * cF - th * uF) / (th * th));
    }
}

int oracle_source(int Q, double tau, double ux, double uy, double Fx, double Fy, double* S) {
    olat L;
    if (build_lattice(Q, &L) || !(tau > 0.5)) return -1;
    guo_source(&L, tau, ux, uy, Fx, Fy, S);
    return 0;
}

/* Collision of one node from its advected populations fadv (after the wall rule): Eq. 16 (with
 * the half-force velocity u = (sum f c + F/2)/rho when a body force g acts, F = rho g along x),
 * Eq. 15 (or its 4th-order continuation), then Eq. 18 with the projection of Eq. 19 (collision 1)
 * or the explicit BGK step of Eq. 14 (collision 0), plus the source S_i when g != 0. */
static void collide(const olat* L, int eq_order, int collision, double tau, const double* fadv, double gx,
                    double* fout) {
    int i, Q = L->Q;
    double feq[OQMAX], fne[OQMAX], S[OQMAX];
    double rho = 0, jx = 0, jy = 0, ux, uy, Fbx, Fby;
    for (i = 0; i < Q; ++i) {
        rho += fadv[i];
        jx += fadv[i] * L->c[i][0];
        jy += fadv[i] * L->c[i][1];
    }
    Fbx = rho * gx;
    Fby = 0.0;
    ux = (jx + 0.5 * Fbx) / rho;
    uy = (jy + 0.5 * Fby) / rho;
    equilibrium(L, eq_order, rho, ux, uy, feq);
    if (collision == 1) project_nonequilibrium(L, fadv, feq, fne);
    for (i = 0; i < Q; ++i) S[i] = 0.0;
    if (gx != 0.0) guo_source(L, tau, ux, uy, Fbx, Fby, S);
    for (i = 0; i < Q; ++i) {
        if (collision == 1)
            fout[i] = feq[i] + (1.0 - 1.0 / tau) * fne[i] + S[i];   /* Eq. 18 */
        else
            fout[i] = fadv[i] - (fadv[i] - feq[i]) / tau + S[i];    /* Eq. 14, explicit step */
    }
}

/* One node's collision for the test suite (same code as the time step). */
int oracle_collide(int Q, int eq_order, int collision, double tau, const double* fadv, double gx, double* fout) {
    olat L;
    if (build_lattice(Q, &L) || (eq_order != 2 && eq_order != 4) || (collision != 0 && collision != 1) ||
        !(tau > 0.5))
        return -1;
    collide(&L, eq_order, collision, tau, fadv, gx, fout);
    return 0;
}

typedef struct {
    int Q;                       /* 9 or 37                                                   */
    int nx, ny;                  /* periodic box; walls are solid labels inside it             */
    double tau;                  /* relaxation time in steps (tau > 1/2)                       */
    double omega;                /* angular frequency of the drive, rad/step                   */
    double u0;                   /* velocity amplitude of the drive                            */
    double rho0;                 /* rest density                                               */
    int eq_order;                /* 2 (Eq. 15) or 4                                            */
    int collision;               /* 0: plain BGK (Eq. 14 discretized), 1: regularized (Eq. 18)  */
    int drive;                   /* 0: label-1 wall moves with U_w = u0 sin(wt) x; 1: body force
                                    g = u0 w cos(wt) x on the fluid, all walls static            */
    const unsigned char* label;  /* ny*nx row-major: 0 fluid, 1 body (force counted), 2 wall    */
    int wall;                    /* 0: bounce-back (Eq. 12); 1: diffuse scattering (Eq. 11)      */
} oracle_params;

static int gcd_int(int a, int b) {
    while (b) { int t = a % b; a = b; b = t; }
    return a; /* gcd(0,0) = 0: the rest population has no link */
}

/* One fluid node of one step, Eqs. 17 -> 16 -> 15 -> 19 -> 18 (or plain BGK), with bounce-back
 * (Eq. 12) on blocked links.  Adds the momentum given to label-1 solids to *Fx, *Fy. */
static void node_update(const olat* L, const oracle_params* p, const double* f, double* fout, int x, int y,
                        double uw, double gx, double* Fx, double* Fy) {
    int Q = L->Q, i, k;
    double fadv[OQMAX];
    const double* fx = f + ((size_t)y * p->nx + x) * Q;
    double th = L->theta;

    /* Eq. 17; links blocked by a solid get Eq. 12 or Eq. 11 below */
    int blocked[OQMAX];
    for (i = 0; i < Q; ++i) {
        int cx = L->c[i][0], cy = L->c[i][1];
        int g = gcd_int(abs(cx), abs(cy)), hit = 0, sx = x, sy = y;
        /* the lattice nodes on the link are x - k c_i/g, k = 1..g (k = g is the pull source);
         * the first solid one met going back from x is the wall the population hits */
        for (k = 1; k <= g; ++k) {
            sx = ((x - k * cx / g) % p->nx + p->nx) % p->nx;
            sy = ((y - k * cy / g) % p->ny + p->ny) % p->ny;
            if (p->label[(size_t)sy * p->nx + sx]) { hit = p->label[(size_t)sy * p->nx + sx]; break; }
        }
        blocked[i] = hit;
        if (!hit) fadv[i] = f[((size_t)sy * p->nx + sx) * Q + i];
    }
    if (p->wall == 0) {
        /* Eq. 12: the node's own opposite population comes back, plus 2 w_i rho0 c_i.U_w / theta */
        for (i = 0; i < Q; ++i) {
            if (!blocked[i]) continue;
            double u_wall = (blocked[i] == 1 && p->drive == 0) ? uw : 0.0;
            fadv[i] = fx[L->opp[i]] + 2.0 * L->w[i] * p->rho0 * (L->c[i][0] * u_wall) / th;
        }
    } else {
        /* Eq. 11: wall Maxwellian at U_w, density from zero net mass flux into each wall */
        int lab;
        for (lab = 1; lab <= 2; ++lab) {
            double u_wall = (lab == 1 && p->drive == 0) ? uw : 0.0, feq1[OQMAX], in = 0.0, den = 0.0, rho_w;
            equilibrium(L, p->eq_order, 1.0, u_wall, 0.0, feq1);
            for (i = 0; i < Q; ++i)
                if (blocked[i] == lab) { in += fx[L->opp[i]]; den += feq1[i]; }
            if (den == 0.0) continue;
            rho_w = in / den;
            for (i = 0; i < Q; ++i)
                if (blocked[i] == lab) fadv[i] = rho_w * feq1[i];
        }
    }
    /* momentum carried into the body by f_opp (velocity -c_i) and out by f_i^adv (velocity c_i) */
    for (i = 0; i < Q; ++i)
        if (blocked[i] == 1) {
            *Fx += -L->c[i][0] * (fx[L->opp[i]] + fadv[i]);
            *Fy += -L->c[i][1] * (fx[L->opp[i]] + fadv[i]);
        }
    collide(L, p->eq_order, p->collision, p->tau, fadv, gx, fout);
}

/* Advance the post-collision state f (ny*nx*Q, full populations, AoS) from step n0 by nsteps
 * steps; force[2k], force[2k+1] receive (Fx, Fy) on the label-1 body during step n0+k, stamped at
 * t = n0 + k + 1/2.  Solid nodes keep their populations.  Returns 0, or -1 on bad arguments. */
int oracle_run(const oracle_params* p, long n0, long nsteps, double* f, double* force, int nthreads) {
    olat L;
    double *tmp, *rowF;
    long n;
    int y;
    size_t N;
    if (!p || !f || !p->label || build_lattice(p->Q, &L)) return -1;
    if (p->nx < 1 || p->ny < 1 || !(p->tau > 0.5) || (p->eq_order != 2 && p->eq_order != 4)) return -1;
    if (p->collision != 0 && p->collision != 1) return -1;
    if (p->drive != 0 && p->drive != 1) return -1;
    if (p->wall != 0 && p->wall != 1) return -1;
    N = (size_t)p->nx * p->ny * L.Q;
    tmp = (double*)malloc(N * sizeof(double));
    rowF = (double*)malloc((size_t)p->ny * 2 * sizeof(double));
    if (!tmp || !rowF) { free(tmp); free(rowF); return -2; }
    (void)nthreads;
    for (n = n0; n < n0 + nsteps; ++n) {
        double t = (double)n + 0.5;
        double uw = p->drive == 0 ? p->u0 * sin(p->omega * t) : 0.0;
        double gx = p->drive == 1 ? p->u0 * p->omega * cos(p->omega * t) : 0.0;
        double Fx = 0.0, Fy = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (y = 0; y < p->ny; ++y) {
            int x, i;
            double fx = 0.0, fy = 0.0;
            for (x = 0; x < p->nx; ++x) {
                size_t node = (size_t)y * p->nx + x;
                if (p->label[node]) {
                    for (i = 0; i < L.Q; ++i) tmp[node * L.Q + i] = f[node * L.Q + i];
                } else {
                    node_update(&L, p, f, tmp + node * L.Q, x, y, uw, gx, &fx, &fy);
                }
            }
            rowF[2 * y] = fx;
            rowF[2 * y + 1] = fy;
        }
        for (y = 0; y < p->ny; ++y) { Fx += rowF[2 * y]; Fy += rowF[2 * y + 1]; }
        if (force) { force[2 * (n - n0)] = Fx; force[2 * (n - n0) + 1] = Fy; }
        memcpy(f, tmp, N * sizeof(double));
    }
    free(tmp);
    free(rowF);
    return 0;
}

/* Number of threads an OpenMP build would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
