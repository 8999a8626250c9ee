/*
 * Spatial operator R(U) of the oracle, written once and instantiated twice by
 * music_oracle.c: with T = double (the oracle proper) and with T = double
 * complex (complex-step differentiation for the exact Jacobian pins).  Every
 * branch is taken on the real part, so the complex instantiation is the exact
 * derivative of the branch-frozen real operator.
 *
 * TEST INFRASTRUCTURE ONLY.  See music_oracle.c for the conventions.
 *
 * What it computes (Sec. 2 of the paper, Eqs. 1-3, staggered grid with
 * upstream linear reconstruction and the van Leer limiter):
 *   R_rho = -div(rho u)
 *   R_E   = -div(rho e u) - p div(u) + div(chi grad T)   (E = rho e)
 *   R_m   = -div(rho u (x) u) - grad p + rho g  (m_d on d-faces)
 * with T = (gamma - 1) e and the photon conductivity chi = 16 sigma T^3 /
 * (3 kappa rho) of Sec. 2 for a Kramers opacity kappa = kappa0 rho T^-3.5,
 * i.e. chi = chi0 T^6.5 / rho^2 (conduction only when g->conduct).
 * Cartesian grids, or 2-D axisymmetric spherical (r, theta) grids where every
 * divergence is (1/V) sum(A F) over the faces of the control volume and the
 * momentum equations carry the geometric terms +rho u_theta^2 / r (radial)
 * and -rho u_r u_theta / r (polar).
 *
 * Required macros: T, RE(x) (real part), SQRT(x), FN(name) (name mangling).
 */

/* van Leer limited slope from the two one-sided differences a, b. */
static T FN(vanleer)(T a, T b)
{
    if (RE(a) * RE(b) > 0.0)
        return (2.0 * a) * b / (a + b);
    return 0.0;
}

/*
 * R(U).  U and R hold nv planes of N = nx*ny*nz values (rho, E, m_x, m_y
 * [, m_z]), x fastest.  m_d[c] sits on the lower d-face of cell c.  On a wall
 * direction w the stored lower wall face (c_w == 0) carries no flux and gets
 * R = 0; the upper wall face is implicit.  Fout, when not NULL, receives the
 * mass fluxes u rho* on the d-faces (one extended-grid array per direction,
 * the flux of the lower d-face of each point) for the passive scalars.
 */
static void FN(spatial_operator_f)(const or_grid *g, const T *U, T *R, T **Fout, T *Aout)
{
    const int nd = g->nd;
    const long N = or_ncells(g);
    or_ext X;
    or_ext_init(&X, g);
    const long M = X.total;

    T *rho = (T *)calloc(M, sizeof(T));
    T *e = (T *)calloc(M, sizeof(T));
    T *p = (T *)calloc(M, sizeof(T));
    T *uf[3], *srho[3], *se[3], *Frho[3], *FE[3], *Phi[3];
    T *su[3][3], *Psi[3][3];
    for (int d = 0; d < 3; d++) {
        uf[d] = srho[d] = se[d] = Frho[d] = FE[d] = Phi[d] = NULL;
        for (int q = 0; q < 3; q++) su[d][q] = Psi[d][q] = NULL;
    }
    for (int d = 0; d < nd; d++) {
        uf[d] = (T *)calloc(M, sizeof(T));
        srho[d] = (T *)calloc(M, sizeof(T));
        se[d] = (T *)calloc(M, sizeof(T));
        Frho[d] = (T *)calloc(M, sizeof(T));
        FE[d] = (T *)calloc(M, sizeof(T));
        Phi[d] = (T *)calloc(M, sizeof(T));
        for (int q = 0; q < nd; q++) {
            su[d][q] = (T *)calloc(M, sizeof(T));
            Psi[d][q] = (T *)calloc(M, sizeof(T));
        }
    }
    T *Erho = (T *)calloc(M, sizeof(T)); /* E on the extended grid */
    T *Tt = NULL, *chi = NULL, *Gc[3] = {NULL, NULL, NULL};
    if (g->conduct) {
        Tt = (T *)calloc(M, sizeof(T));
        chi = (T *)calloc(M, sizeof(T));
        for (int d = 0; d < nd; d++) Gc[d] = (T *)calloc(M, sizeof(T));
    }
    const int sph = (g->geom == OR_GEOM_SPHERICAL);

    const double gm1 = g->gamma - 1.0;

    /* --- a1: interior values, then ghost layers direction by direction --- */
    OR_PAR
    for (long c = 0; c < N; c++) {
        long x = or_ext_of_cell(&X, g, c);
        rho[x] = U[c];
        Erho[x] = U[N + c];
    }
    for (int d = 0; d < nd; d++) {
        OR_PAR
        for (long x = 0; x < M; x++) {
            int ix[3];
            or_ext_coords(&X, x, ix);
            int a = ix[d];
            if (a >= 0 && a < g->n[d]) continue; /* not a ghost along d */
            /* skip points that are ghosts along a later direction: they are
               filled when that direction is processed */
            int later = 0;
            for (int q = d + 1; q < nd; q++)
                if (ix[q] < 0 || ix[q] >= g->n[q]) later = 1;
            if (later) continue;
            int src[3] = {ix[0], ix[1], ix[2]};
            if (g->bc[d] == OR_BC_PERIODIC) {
                src[d] = ((a % g->n[d]) + g->n[d]) % g->n[d];
                long s = or_ext_index(&X, src);
                rho[x] = rho[s];
                Erho[x] = Erho[s];
            } else if (g->wall_scalar[d] == OR_WALL_MIRROR) {
                src[d] = (a < 0) ? (-1 - a) : (2 * g->n[d] - 1 - a);
                long s = or_ext_index(&X, src);
                rho[x] = rho[s];
                Erho[x] = Erho[s];
            } else {
                /* hydrostatic ghost: T extrapolated linearly, rho from the
                   discrete balance (p_b - p_g) = +-dx g (rho_b + rho_g)/2
                   across the wall face, p = rho T.  Only the first ghost
                   layer enters any flux; deeper layers copy it. */
                const int lower = (a < 0);
                const int b0 = lower ? 0 : g->n[d] - 1;
                const int b1 = lower ? 1 : g->n[d] - 2;
                int i0[3] = {ix[0], ix[1], ix[2]}, i1[3] = {ix[0], ix[1], ix[2]};
                i0[d] = b0;
                i1[d] = b1;
                long s0 = or_ext_index(&X, i0), s1 = or_ext_index(&X, i1);
                T T0 = gm1 * Erho[s0] / rho[s0];
                T T1 = gm1 * Erho[s1] / rho[s1];
                T Tg = 2.0 * T0 - T1;
                double hs = 0.5 * g->dx[d] * or_gface(g, d, lower ? 0 : g->n[d]);
                T rg = lower ? rho[s0] * (T0 - hs) / (Tg + hs)
                             : rho[s0] * (T0 + hs) / (Tg - hs);
                rho[x] = rg;
                Erho[x] = rg * Tg / gm1;
            }
        }
    }
    OR_PAR
    for (long x = 0; x < M; x++) {
        e[x] = Erho[x] / rho[x];
        p[x] = gm1 * Erho[x];
    }
    if (g->conduct) {
        /* temperature and conductivity per cell; gradient flux chi dT/dn on
           every d-face (arithmetic mean of the two cells' chi); wall faces
           carry the prescribed flux or none */
        OR_PAR
        for (long x = 0; x < M; x++) {
            Tt[x] = gm1 * e[x];
            T t3 = Tt[x] * Tt[x] * Tt[x];
            chi[x] = g->chi0 * (t3 * t3 * SQRT(Tt[x])) / (rho[x] * rho[x]);
        }
        for (int d = 0; d < nd; d++) {
            const long s = X.stride[d];
            OR_PAR
            for (long x = 0; x < M; x++) {
                int ix[3];
                or_ext_coords(&X, x, ix);
                if (!or_ext_has(&X, ix, d, -1)) continue;
                if (g->bc[d] == OR_BC_WALL && (ix[d] == 0 || ix[d] == g->n[d])) {
                    double G = 0.0;
                    if (g->flux_wall[d]) {
                        G = g->lum;
                        if (sph && d == 0) {
                            double rf = or_r(g, ix[0]);
                            G = G / (rf * rf);
                        }
                    }
                    Gc[d][x] = G;
                    continue;
                }
                double h = sph ? or_sph_h(g, d, ix[0]) : g->dx[d];
                Gc[d][x] = 0.5 * (chi[x - s] + chi[x]) * (Tt[x] - Tt[x - s]) / h;
            }
        }
    }

    /* --- face velocities: interior faces from m / (mean of the two cells) --- */
    for (int d = 0; d < nd; d++) {
        OR_PAR
        for (long c = 0; c < N; c++) {
            long x = or_ext_of_cell(&X, g, c);
            int ix[3];
            or_ext_coords(&X, x, ix);
            if (g->bc[d] == OR_BC_WALL && ix[d] == 0) {
                uf[d][x] = 0.0;
                continue;
            }
            long xl = x - X.stride[d];
            T rbar = 0.5 * (rho[xl] + rho[x]);
            uf[d][x] = U[(2 + d) * N + c] / rbar;
        }
    }
    /* ghost face velocities, direction by direction */
    for (int w = 0; w < nd; w++) {
        OR_PAR
        for (long x = 0; x < M; x++) {
            int ix[3];
            or_ext_coords(&X, x, ix);
            int a = ix[w];
            if (a >= 0 && a < g->n[w]) continue;
            int later = 0;
            for (int q = w + 1; q < nd; q++)
                if (ix[q] < 0 || ix[q] >= g->n[q]) later = 1;
            if (later) continue;
            for (int d = 0; d < nd; d++) {
                int src[3] = {ix[0], ix[1], ix[2]};
                if (g->bc[w] == OR_BC_PERIODIC) {
                    src[w] = ((a % g->n[w]) + g->n[w]) % g->n[w];
                    uf[d][x] = uf[d][or_ext_index(&X, src)];
                } else if (d == w) {
                    /* normal velocity on w-faces: zero on the wall faces,
                       odd reflection beyond them */
                    const int n = g->n[w];
                    if (a == n) {
                        uf[d][x] = 0.0;
                    } else {
                        src[w] = (a < 0) ? -a : 2 * n - a;
                        uf[d][x] = -uf[d][or_ext_index(&X, src)];
                    }
                } else {
                    /* tangential velocity: stress-free, even reflection */
                    src[w] = (a < 0) ? (-1 - a) : (2 * g->n[w] - 1 - a);
                    uf[d][x] = uf[d][or_ext_index(&X, src)];
                }
            }
        }
    }

    /* --- limited slopes --- */
    for (int d = 0; d < nd; d++) {
        const long s = X.stride[d];
        OR_PAR
        for (long x = 0; x < M; x++) {
            int ix[3];
            or_ext_coords(&X, x, ix);
            if (!or_ext_has(&X, ix, d, -1) || !or_ext_has(&X, ix, d, +1)) continue;
            srho[d][x] = FN(vanleer)(rho[x] - rho[x - s], rho[x + s] - rho[x]);
            se[d][x] = FN(vanleer)(e[x] - e[x - s], e[x + s] - e[x]);
            for (int q = 0; q < nd; q++) /* slope of u_q along d, on q-faces */
                su[q][d][x] = FN(vanleer)(uf[q][x] - uf[q][x - s], uf[q][x + s] - uf[q][x]);
        }
    }

    /* --- mass and internal-energy fluxes on d-faces (upwind reconstruction) --- */
    for (int d = 0; d < nd; d++) {
        const long s = X.stride[d];
        OR_PAR
        for (long x = 0; x < M; x++) {
            int ix[3];
            or_ext_coords(&X, x, ix);
            if (!or_ext_has(&X, ix, d, -2) || !or_ext_has(&X, ix, d, +1)) continue;
            T u = uf[d][x];
            T rs, es;
            if (RE(u) >= 0.0) {
                rs = rho[x - s] + 0.5 * srho[d][x - s];
                es = e[x - s] + 0.5 * se[d][x - s];
            } else {
                rs = rho[x] - 0.5 * srho[d][x];
                es = e[x] - 0.5 * se[d][x];
            }
            Frho[d][x] = u * rs;
            FE[d][x] = Frho[d][x] * es;
        }
    }

    /* --- momentum fluxes --- */
    for (int d = 0; d < nd; d++) {
        const long s = X.stride[d];
        /* flux of m_d along d at cell centres */
        OR_PAR
        for (long x = 0; x < M; x++) {
            int ix[3];
            or_ext_coords(&X, x, ix);
            if (!or_ext_has(&X, ix, d, -2) || !or_ext_has(&X, ix, d, +2)) continue;
            T fm = 0.5 * (Frho[d][x] + Frho[d][x + s]);
            T us = (RE(fm) >= 0.0) ? uf[d][x] + 0.5 * su[d][d][x]
                                   : uf[d][x + s] - 0.5 * su[d][d][x + s];
            Phi[d][x] = fm * us;
        }
        /* flux of m_d along q (q != d) on the (d,q) edges at the lower
           d- and q-faces of cell x */
        for (int q = 0; q < nd; q++) {
            if (q == d) continue;
            const long t = X.stride[q];
            OR_PAR
            for (long x = 0; x < M; x++) {
                int ix[3];
                or_ext_coords(&X, x, ix);
                if (!or_ext_has(&X, ix, d, -1) || !or_ext_has(&X, ix, q, -2) ||
                    !or_ext_has(&X, ix, q, +1))
                    continue;
                T fm = 0.5 * (Frho[q][x - s] + Frho[q][x]);
                T us = (RE(fm) >= 0.0) ? uf[d][x - t] + 0.5 * su[d][q][x - t]
                                       : uf[d][x] - 0.5 * su[d][q][x];
                Psi[d][q][x] = fm * us;
            }
        }
    }

    /* --- residual assembly on the interior --- */
    OR_PAR
    for (long c = 0; c < (sph ? 0 : N); c++) {
        long x = or_ext_of_cell(&X, g, c);
        int ix[3];
        or_ext_coords(&X, x, ix);
        T accr = 0.0, acce = 0.0, divu = 0.0;
        for (int d = 0; d < nd; d++) {
            const long s = X.stride[d];
            accr += (Frho[d][x + s] - Frho[d][x]) / g->dx[d];
            acce += (FE[d][x + s] - FE[d][x]) / g->dx[d];
            divu += (uf[d][x + s] - uf[d][x]) / g->dx[d];
        }
        R[c] = -accr;
        R[N + c] = -acce - p[x] * divu;
        if (g->conduct) {
            T cond = 0.0;
            for (int d = 0; d < nd; d++) {
                const long s = X.stride[d];
                cond += (Gc[d][x + s] - Gc[d][x]) / g->dx[d];
            }
            R[N + c] = R[N + c] + cond;
        }
        if (Aout) {
            /* the magnitude of every term the residual of this cell sums */
            T ar = 0.0, ae = 0.0, au = 0.0;
            for (int d = 0; d < nd; d++) {
                const long s = X.stride[d];
                ar += (TABS(Frho[d][x + s]) + TABS(Frho[d][x])) / g->dx[d];
                ae += (TABS(FE[d][x + s]) + TABS(FE[d][x])) / g->dx[d];
                au += (TABS(uf[d][x + s]) + TABS(uf[d][x])) / g->dx[d];
                if (g->conduct) ae += (TABS(Gc[d][x + s]) + TABS(Gc[d][x])) / g->dx[d];
            }
            Aout[c] = ar;
            Aout[N + c] = ae + TABS(p[x]) * au;
        }
        for (int d = 0; d < nd; d++) {
            if (g->bc[d] == OR_BC_WALL && ix[d] == 0) {
                R[(2 + d) * N + c] = 0.0;
                continue;
            }
            const long s = X.stride[d];
            T acc = 0.0;
            for (int q = 0; q < nd; q++) {
                if (q == d)
                    acc += (Phi[d][x] - Phi[d][x - s]) / g->dx[d];
                else
                    acc += (Psi[d][q][x + X.stride[q]] - Psi[d][q][x]) / g->dx[q];
            }
            T rbar = 0.5 * (rho[x - s] + rho[x]);
            R[(2 + d) * N + c] = (-acc - (p[x] - p[x - s]) / g->dx[d]) + rbar * g->g[d];
            if (Aout) {
                T am = 0.0;
                for (int q = 0; q < nd; q++) {
                    if (q == d)
                        am += (TABS(Phi[d][x]) + TABS(Phi[d][x - s])) / g->dx[d];
                    else
                        am += (TABS(Psi[d][q][x + X.stride[q]]) + TABS(Psi[d][q][x])) / g->dx[q];
                }
                Aout[(2 + d) * N + c] = am + (TABS(p[x]) + TABS(p[x - s])) / g->dx[d] + TABS(rbar * g->g[d]);
            }
        }
        if (Aout)
            for (int d = 0; d < nd; d++)
                if (g->bc[d] == OR_BC_WALL && ix[d] == 0) Aout[(2 + d) * N + c] = 0.0;
    }
    /* spherical (r, theta): area-weighted divergences over each control volume */
    OR_PAR
    for (long c = 0; c < (sph ? N : 0); c++) {
        long x = or_ext_of_cell(&X, g, c);
        int ix[3];
        or_ext_coords(&X, x, ix);
        const int i = ix[0], j = ix[1];
        const long s0 = X.stride[0], s1 = X.stride[1];
        const double V = or_sph_vol(g, i, j);
        const double Arm = or_sph_area(g, 0, i, j), Arp = or_sph_area(g, 0, i + 1, j);
        const double Atm = or_sph_area(g, 1, i, j), Atp = or_sph_area(g, 1, i, j + 1);
        T fr = (Arp * Frho[0][x + s0] - Arm * Frho[0][x]) + (Atp * Frho[1][x + s1] - Atm * Frho[1][x]);
        T fe = (Arp * FE[0][x + s0] - Arm * FE[0][x]) + (Atp * FE[1][x + s1] - Atm * FE[1][x]);
        T du = (Arp * uf[0][x + s0] - Arm * uf[0][x]) + (Atp * uf[1][x + s1] - Atm * uf[1][x]);
        R[c] = -fr / V;
        R[N + c] = -fe / V - p[x] * (du / V);
        if (g->conduct) {
            T cd = (Arp * Gc[0][x + s0] - Arm * Gc[0][x]) + (Atp * Gc[1][x + s1] - Atm * Gc[1][x]);
            R[N + c] = R[N + c] + cd / V;
        }
        if (Aout) {
            Aout[c] = (Arp * TABS(Frho[0][x + s0]) + Arm * TABS(Frho[0][x]) + Atp * TABS(Frho[1][x + s1]) +
                       Atm * TABS(Frho[1][x])) / V;
            T ae = (Arp * TABS(FE[0][x + s0]) + Arm * TABS(FE[0][x]) + Atp * TABS(FE[1][x + s1]) +
                    Atm * TABS(FE[1][x])) / V;
            ae += TABS(p[x]) * ((Arp * TABS(uf[0][x + s0]) + Arm * TABS(uf[0][x]) + Atp * TABS(uf[1][x + s1]) +
                                 Atm * TABS(uf[1][x])) / V);
            if (g->conduct)
                ae += (Arp * TABS(Gc[0][x + s0]) + Arm * TABS(Gc[0][x]) + Atp * TABS(Gc[1][x + s1]) +
                       Atm * TABS(Gc[1][x])) / V;
            Aout[N + c] = ae;
            Aout[2 * N + c] = 0.0;
            Aout[3 * N + c] = 0.0;
        }
        const double ctj = cos(or_th(g, j)), ctj1 = cos(or_th(g, j + 1));
        /* radial momentum on r-face i: control volume r_{i-1/2}..r_{i+1/2} */
        if (g->bc[0] == OR_BC_WALL && i == 0) {
            R[2 * N + c] = 0.0;
        } else {
            const double rm = or_r(g, i - 0.5), rp = or_r(g, i + 0.5), rf = or_r(g, i);
            const double Vr = (rp * rp * rp - rm * rm * rm) / 3.0 * (ctj - ctj1);
            const double Acp = rp * rp * (ctj - ctj1), Acm = rm * rm * (ctj - ctj1);
            const double Em = 0.5 * (rp * rp - rm * rm) * sin(or_th(g, j));
            const double Ep = 0.5 * (rp * rp - rm * rm) * sin(or_th(g, j + 1));
            T acc = (Acp * Phi[0][x] - Acm * Phi[0][x - s0]) + (Ep * Psi[0][1][x + s1] - Em * Psi[0][1][x]);
            T rbar = 0.5 * (rho[x - s0] + rho[x]);
            T ut = 0.25 * ((uf[1][x - s0] + uf[1][x]) + (uf[1][x - s0 + s1] + uf[1][x + s1]));
            R[2 * N + c] = ((-acc / Vr - (p[x] - p[x - s0]) / g->dx[0]) + rbar * ut * ut / rf) +
                           rbar * or_gface(g, 0, i);
            if (Aout)
                Aout[2 * N + c] = (Acp * TABS(Phi[0][x]) + Acm * TABS(Phi[0][x - s0]) + Ep * TABS(Psi[0][1][x + s1]) +
                                   Em * TABS(Psi[0][1][x])) / Vr +
                                  (TABS(p[x]) + TABS(p[x - s0])) / g->dx[0] + TABS(rbar * ut * ut / rf) +
                                  TABS(rbar * or_gface(g, 0, i));
        }
        /* polar momentum on theta-face j: control volume theta_{j-1/2}..theta_{j+1/2} */
        if (g->bc[1] == OR_BC_WALL && j == 0) {
            R[3 * N + c] = 0.0;
        } else {
            const double ra = or_r(g, i), rb = or_r(g, i + 1), rc = or_r(g, i + 0.5);
            const double cm = cos(or_th(g, j - 0.5)), cp = cos(or_th(g, j + 0.5));
            const double Vt = (rb * rb * rb - ra * ra * ra) / 3.0 * (cm - cp);
            const double Bp = 0.5 * (rb * rb - ra * ra) * sin(or_th(g, j + 0.5));
            const double Bm = 0.5 * (rb * rb - ra * ra) * sin(or_th(g, j - 0.5));
            const double Fa = ra * ra * (cm - cp), Fb = rb * rb * (cm - cp);
            T acc = (Fb * Psi[1][0][x + s0] - Fa * Psi[1][0][x]) + (Bp * Phi[1][x] - Bm * Phi[1][x - s1]);
            T rbar = 0.5 * (rho[x - s1] + rho[x]);
            T ur = 0.25 * ((uf[0][x - s1] + uf[0][x]) + (uf[0][x - s1 + s0] + uf[0][x + s0]));
            R[3 * N + c] = ((-acc / Vt - (p[x] - p[x - s1]) / (rc * g->dx[1])) - rbar * ur * uf[1][x] / rc) +
                           rbar * g->g[1];
            if (Aout)
                Aout[3 * N + c] = (Fb * TABS(Psi[1][0][x + s0]) + Fa * TABS(Psi[1][0][x]) + Bp * TABS(Phi[1][x]) +
                                   Bm * TABS(Phi[1][x - s1])) / Vt +
                                  (TABS(p[x]) + TABS(p[x - s1])) / (rc * g->dx[1]) + TABS(rbar * ur * uf[1][x] / rc) +
                                  TABS(rbar * g->g[1]);
        }
    }

    if (Fout)
        for (int d = 0; d < nd; d++) memcpy(Fout[d], Frho[d], M * sizeof(T));
    free(rho); free(e); free(p); free(Erho); free(Tt); free(chi);
    for (int d = 0; d < nd; d++) free(Gc[d]);
    for (int d = 0; d < nd; d++) {
        free(uf[d]); free(srho[d]); free(se[d]); free(Frho[d]); free(FE[d]); free(Phi[d]);
        for (int q = 0; q < nd; q++) { free(su[d][q]); free(Psi[d][q]); }
    }
}

static void FN(spatial_operator)(const or_grid *g, const T *U, T *R) { FN(spatial_operator_f)(g, U, R, NULL, NULL); }

/*
 * Passive scalars (Sec. 2.2): S_i(q) = -div(c_i rho u) for the partial
 * densities q_i = c_i rho of ns scalars (ns planes of N values), with the
 * fluid frozen: rho (N cell densities) and the mass fluxes Fr[d] (extended
 * grid, lower d-face of each point) of the fluid state.  The scalar flux on
 * a face is the mass flux times c_i reconstructed upwind with the van Leer
 * limiter, the form of the internal-energy flux, so a uniform c_i is carried
 * exactly like the density.  Ghost values of c_i: periodic wrap, mirror at
 * walls (wall faces carry no mass flux).  Cartesian grids.
 */
static void FN(scalar_operator)(const or_grid *g, const double *rho, double *const *Fr, const T *q, int ns, T *S)
{
    const int nd = g->nd;
    const long N = or_ncells(g);
    or_ext X;
    or_ext_init(&X, g);
    const long M = X.total;
    T *c = (T *)calloc(M, sizeof(T));
    T *sc = (T *)calloc(M, sizeof(T));
    T *Fs[3] = {NULL, NULL, NULL};
    for (int d = 0; d < nd; d++) Fs[d] = (T *)calloc(M, sizeof(T));
    for (int i = 0; i < ns; i++) {
        OR_PAR
        for (long k = 0; k < N; k++) c[or_ext_of_cell(&X, g, k)] = q[(long)i * N + k] / rho[k];
        for (int d = 0; d < nd; d++) {
            OR_PAR
            for (long x = 0; x < M; x++) {
                int ix[3];
                or_ext_coords(&X, x, ix);
                int a = ix[d];
                if (a >= 0 && a < g->n[d]) continue;
                int later = 0;
                for (int w = d + 1; w < nd; w++)
                    if (ix[w] < 0 || ix[w] >= g->n[w]) later = 1;
                if (later) continue;
                int src[3] = {ix[0], ix[1], ix[2]};
                if (g->bc[d] == OR_BC_PERIODIC)
                    src[d] = ((a % g->n[d]) + g->n[d]) % g->n[d];
                else
                    src[d] = (a < 0) ? (-1 - a) : (2 * g->n[d] - 1 - a);
                c[x] = c[or_ext_index(&X, src)];
            }
        }
        for (int d = 0; d < nd; d++) {
            const long s = X.stride[d];
            OR_PAR
            for (long x = 0; x < M; x++) {
                int ix[3];
                or_ext_coords(&X, x, ix);
                sc[x] = 0.0;
                if (!or_ext_has(&X, ix, d, -1) || !or_ext_has(&X, ix, d, +1)) continue;
                sc[x] = FN(vanleer)(c[x] - c[x - s], c[x + s] - c[x]);
            }
            OR_PAR
            for (long x = 0; x < M; x++) {
                int ix[3];
                or_ext_coords(&X, x, ix);
                Fs[d][x] = 0.0;
                if (!or_ext_has(&X, ix, d, -2) || !or_ext_has(&X, ix, d, +1)) continue;
                const double f = Fr[d][x];
                const T cs = (f >= 0.0) ? c[x - s] + 0.5 * sc[x - s] : c[x] - 0.5 * sc[x];
                Fs[d][x] = f * cs;
            }
        }
        OR_PAR
        for (long k = 0; k < N; k++) {
            const long x = or_ext_of_cell(&X, g, k);
            T acc = 0.0;
            for (int d = 0; d < nd; d++) {
                const long s = X.stride[d];
                acc += (Fs[d][x + s] - Fs[d][x]) / g->dx[d];
            }
            S[(long)i * N + k] = -acc;
        }
    }
    free(c);
    free(sc);
    for (int d = 0; d < nd; d++) free(Fs[d]);
}
