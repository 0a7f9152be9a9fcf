/*
 * FP64 CPU oracle of the combined lattice Boltzmann / immersed boundary method of
 * Coclite et al., "Kinematic and Dynamic Forcing Strategies for Predicting the
 * Transport of Inertial Capsules via a combined Lattice Boltzmann - Immersed Boundary
 * Method" (arXiv:1903.03356).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously-correct statement
 * of what the GPU library computes. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it. It shares no code, header, table or constant
 * with the CUDA library; the library never calls it.
 *
 * Style: scalar loops in the order and notation of the paper, double precision, no
 * blocking, fusion or reordering beyond what each equation states. Built with
 * -O2 -ffp-contract=off so that x86 and Arm hosts give identical bits.
 *
 * Units: dx = dt = 1, rho_0 = 1, c_s^2 = 1/3, nu = (tau - 1/2)/3. Lattice node (i, j)
 * sits at (x, y) = (i, j). With walls, half-way bounce-back walls sit at y = -1/2 and
 * y = ny - 1/2 (channel height H = ny). x is periodic, or open: a known-velocity inlet
 * at column x = 0 and a known-density outlet at x = nx - 1 (Zou and He, reading R26).
 *
 * Readings of the paper where it is silent, ambiguous or garbled (each also listed in
 * the design notes of the repository):
 *   R1  Eq. 7 prints the forcing term F_i where the body force f_ib is meant:
 *       rho u = sum_i f_i e_i + f_ib / 2 (standard Guo form). The collision uses the
 *       force of its own step; the fields read back and the Kinematic interpolation use
 *       the last spread force.
 *   R1d In the Dynamic scheme the IB force of a step is what is being determined (the
 *       direct forcing of Favier et al., which Section 2.3 names): every interpolation of
 *       that scheme (U of step 1, the probes of Eq. 15-16 and Eq. 17-18) takes the velocity
 *       of the populations before any IB force, rho u = sum_i f_i e_i + g / 2.
 *   R2  Boundaries: half-way bounce-back with wall velocity; the correction uses the
 *       reference density rho_0 = 1 (keeps mass exactly conserved and is linear).
 *   R3  Markers are the membrane vertices; element quantities go half to each vertex.
 *   R4  Spreading coefficient: Kinematic c_v = 1; Dynamic c_l = rho_0 (l_left+l_right)/2
 *       with current element lengths.
 *   R5  MLS: support centre = nearest node floor(x + 1/2); 3x3 support; linear basis
 *       written about the evaluation point, p = [1, x_k - x, y_k - y] (the same fit,
 *       translated); the velocity gradient is the fitted linear coefficient.
 *   R6  Bending: theta_v = signed turning angle atan2(a x b, a . b) of the incoming
 *       edge a and outgoing edge b; energy k_b (1 - cos(theta - theta_0)), whose
 *       derivative gives the k_b sin(theta - theta_0) factor of Eq. 13.
 *   R7  Green's theorem area A = 1/2 sum (x_i y_{i+1} - x_{i+1} y_i); each end node of
 *       an element receives half of F^a_l; counter-clockwise rings, n+ = (dy, -dx)/l.
 *   R10 Eq. 25: the interpolated velocity is taken at the latest positions X^n.
 *   R11 Eq. 23: the tentative velocity xdot_0(t) is the fluid velocity at time t, the U of
 *       step 1 (interpolated at X^n before the fluid update), as the Verlet form
 *       x(t + dt) = x(t) + v(t) dt + a(t) dt^2 / 2 has it. (Interpolating it after the
 *       update instead makes the step-1 forcing u_v - U grow with the fluid's acceleration
 *       at the marker, and the coupled step is then unstable even with no membrane force.)
 *   R12 viscous stress tau = rho nu (grad u + grad u^T), pressure p = rho / 3.
 *   R15 Taylor D from the eigenvalues of the polygon's area second-moment tensor.
 *   R23 Capsule-capsule repulsion (Section 3.4, Eq. 27): a vertex feels every vertex of
 *       every other ring closer than a cut-off r_c (the paper gives the force law and
 *       that it holds the separation near dx, but no range); x (and y without walls)
 *       distances are minimum images on the periodic lattice.
 *   R24 The normal at a vertex is the normalised sum of the outward unit normals
 *       (dy, -dx)/l of the two elements meeting there; Eq. 27 acts along its negative.
 *   R26 Open channel (Section 2.1, boundaries of Zou and He; Section 3.2 inlet profile
 *       and outlet pressure): on the pre-collision populations of the inlet column the
 *       three populations entering from x < 0 are rebuilt so that the node has the
 *       prescribed velocity (u_in(y), 0); on the outlet column those entering from
 *       x > nx - 1 so that it has density rho_out and zero y-velocity. Closure: mass and
 *       normal momentum fix rho (inlet) or u_x (outlet); the non-equilibrium part
 *       bounces back along the normal, f_1 - f_1^eq = f_3 - f_3^eq; the diagonals carry
 *       the tangential non-equilibrium momentum, f_5^neq - f_7^neq = -(f_2^neq -
 *       f_4^neq)/2 and f_8^neq - f_6^neq = +(f_2^neq - f_4^neq)/2. With the Guo force F
 *       the known momentum is rho u - F/2 and the equilibria are taken at the velocity
 *       of that momentum. The whole column is closed, the wall rows included (their
 *       wall-crossing populations are bounced back first). Supports of markers and
 *       probes must stay inside columns 1 .. nx - 2, so the open columns carry only the
 *       uniform force g; distances along x are not periodic.
 *   R27 Rigid particle (Section 2.3.1): a ring of markers fixed in the body frame, X_v =
 *       c + R(theta) r_v with c the area centroid of the initial ring and r_v = X_v^0 -
 *       c^0. In the Dynamic coupling (Section 2.3.2 steps 1-3) its markers' desired
 *       velocity is the rigid-body velocity u + omega x (X_v - c).
 *   R28 Eq. 17-18: the fluid load is the outer probes' traction (tau+ . n+ - p+ n+) l_l of
 *       every element (no inner fluid), evaluated at X^n after the fluid update (as R11),
 *       with the lever arm r_l from c to the element centroid; the Eq. 27 repulsion on the
 *       markers (when on) adds its sum and moment.
 *   R29 Eq. 19-20 with u(t) -> u^{n+1}, u(t - dt) -> u^n, u(t - 2 dt) -> u^{n-1} and the
 *       acceleration of the current load; the paper prints no position update, so c and
 *       theta take the same second-order backward form as Eq. 24-25:
 *       c^{n+1} = 2/3 (2 c^n - c^{n-1}/2 + u^{n+1} dt), likewise theta. At rest history
 *       (u^{-1} = u^0, c^{-1} = c^0 - u^0 dt, theta^{-1} = theta^0 - omega^0 dt).
 *   R30 Rigid particles exist only in the Dynamic scheme (the Kinematic scheme moves
 *       markers with the fluid); a Kinematic step with one present is refused.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_SUPPORT 5
#define ORC_ERR_STATE 7

/* ---------------------------------------------------------------------------------- */
/* D2Q9 velocity set (Eq. 3) and weights (Section 2.1).                                  */
/* ---------------------------------------------------------------------------------- */
static const int ex_[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey_[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double w_[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int opp_[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

typedef struct {
    int nx, ny;
    int walls;          /* 0: periodic in y; 1: half-way bounce-back walls in y     */
    double u_bottom;    /* x-velocity of the wall at y = -1/2                        */
    double u_top;       /* x-velocity of the wall at y = ny - 1/2                    */
    double tau;         /* BGK relaxation time                                       */
    double gx, gy;      /* uniform body-force density added to f_ib everywhere       */
    int inflow;         /* 0: periodic in x; 1: open inlet and outlet columns (R26)  */
    double rho_out;     /* outlet density                                            */
    const double* u_in; /* inlet x-velocity of every row (ny values)                 */
} orc_lattice;

/* index of population i at node (x, y) */
static size_t fidx(const orc_lattice* L, int i, int x, int y) {
    return ((size_t)i * (size_t)L->ny + (size_t)y) * (size_t)L->nx + (size_t)x;
}
static size_t nidx(const orc_lattice* L, int x, int y) {
    return (size_t)y * (size_t)L->nx + (size_t)x;
}
static int wrap(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Eq. 2: Maxwell-Boltzmann equilibrium with c_s^2 = 1/3. */
void orc_feq(double rho, double ux, double uy, double feq[9]) {
    const double cs2 = 1.0 / 3.0;
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double eu = ex_[i] * ux + ey_[i] * uy;
        feq[i] = w_[i] * rho * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - usq / (2.0 * cs2));
    }
}

/* Total body force at a node: uniform g plus the immersed-boundary field (may be NULL). */
static void node_force(const orc_lattice* L, const double* fib, size_t n, double* Fx, double* Fy) {
    *Fx = L->gx;
    *Fy = L->gy;
    if (fib) {
        size_t N = (size_t)L->nx * (size_t)L->ny;
        *Fx += fib[n];
        *Fy += fib[N + n];
    }
}

/* Eq. 6 and Eq. 7 (reading R1) at one node. */
static void node_macros(const orc_lattice* L, const double* f, const double* fib, int x, int y,
                        double* rho, double* ux, double* uy) {
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < 9; i++) {
        double fi = f[fidx(L, i, x, y)];
        r += fi;
        mx += fi * ex_[i];
        my += fi * ey_[i];
    }
    double Fx, Fy;
    node_force(L, fib, nidx(L, x, y), &Fx, &Fy);
    *rho = r;
    *ux = (mx + 0.5 * Fx) / r;
    *uy = (my + 0.5 * Fy) / r;
}

/* Density and velocity fields (Eq. 6-7); fib holds fx[N] then fy[N] or is NULL. */
void orc_macros(const orc_lattice* L, const double* f, const double* fib, double* rho,
                double* ux, double* uy) {
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t n = nidx(L, x, y);
            node_macros(L, f, fib, x, y, &rho[n], &ux[n], &uy[n]);
        }
}

/*
 * Zou-He closure of the open columns (reading R26) on the pre-collision populations f:
 * column x = 0 gets velocity (u_in[y], 0), column x = nx - 1 density rho_out and zero
 * y-velocity. The open columns carry only the uniform force g.
 */
void orc_open_boundaries(const orc_lattice* L, double* f) {
    if (!L->inflow) return;
    const double Fx = L->gx, Fy = L->gy;
    for (int side = 0; side < 2; side++) {
        const int x = side == 0 ? 0 : L->nx - 1;
        for (int y = 0; y < L->ny; y++) {
            double fi[9], feq[9];
            for (int i = 0; i < 9; i++) fi[i] = f[fidx(L, i, x, y)];
            double rho, jx;
            const double jy = -0.5 * Fy;   /* v = 0: rho v - F_y/2 */
            if (side == 0) {
                /* unknown: 1, 5, 8. Mass: rho = K + (f1 + f5 + f8); normal momentum:
                 * (f1 + f5 + f8) - (f3 + f6 + f7) = rho u - F_x/2. */
                const double u = L->u_in[y];
                const double K = fi[0] + fi[2] + fi[4] + fi[3] + fi[6] + fi[7];
                rho = (K + fi[3] + fi[6] + fi[7] - 0.5 * Fx) / (1.0 - u);
                jx = rho * u - 0.5 * Fx;
            } else {
                /* unknown: 3, 6, 7. Mass fixes the unknown sum, normal momentum follows. */
                rho = L->rho_out;
                const double K = fi[0] + fi[2] + fi[4] + fi[1] + fi[5] + fi[8];
                jx = (fi[1] + fi[5] + fi[8]) - (rho - K);
            }
            orc_feq(rho, jx / rho, jy / rho, feq);
            const double nt = (fi[2] - feq[2]) - (fi[4] - feq[4]);   /* tangential non-equilibrium */
            if (side == 0) {
                fi[1] = fi[3] + (feq[1] - feq[3]);
                fi[5] = fi[7] + (feq[5] - feq[7]) - 0.5 * nt;
                fi[8] = fi[6] + (feq[8] - feq[6]) + 0.5 * nt;
            } else {
                fi[3] = fi[1] - (feq[1] - feq[3]);
                fi[7] = fi[5] - (feq[5] - feq[7]) + 0.5 * nt;
                fi[6] = fi[8] - (feq[8] - feq[6]) - 0.5 * nt;
            }
            for (int i = 0; i < 9; i++) f[fidx(L, i, x, y)] = fi[i];
        }
    }
}

/*
 * One lattice update, Eq. 4 with the forcing term of Eq. 5: every node collides
 * (BGK, Eq. 1-2) with the Guo term built from the total force g + f_ib, then every
 * post-collision population streams to x + e_i. A population that would cross a
 * wall returns to its own node in the opposite direction, corrected by
 * -2 w_i rho_0 (e_i . u_w) / c_s^2 (reading R2). On an open channel the populations
 * that would enter through the inlet or outlet column are then rebuilt (R26). f is
 * pre-collision at time t, fnew receives pre-collision populations at t + 1.
 */
void orc_collide_stream(const orc_lattice* L, const double* f, const double* fib, double* fnew) {
    const double tau = L->tau;
    const double cs2 = 1.0 / 3.0;
    /* Rows are independent (each node writes its own streamed populations), so the
     * all-core build (-fopenmp) splits them over threads with identical results; the
     * plain build ignores the pragma. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < L->ny; y++) {
        for (int x = 0; x < L->nx; x++) {
            double rho, ux, uy, Fx, Fy, feq[9];
            node_macros(L, f, fib, x, y, &rho, &ux, &uy);
            node_force(L, fib, nidx(L, x, y), &Fx, &Fy);
            orc_feq(rho, ux, uy, feq);
            for (int i = 0; i < 9; i++) {
                /* Eq. 5 */
                double eu = ex_[i] * ux + ey_[i] * uy;
                double bx = (ex_[i] - ux) / cs2 + eu / (cs2 * cs2) * ex_[i];
                double by = (ey_[i] - uy) / cs2 + eu / (cs2 * cs2) * ey_[i];
                double Fi = (1.0 - 1.0 / (2.0 * tau)) * w_[i] * (bx * Fx + by * Fy);
                /* Eq. 4 */
                double fpost = f[fidx(L, i, x, y)] - (f[fidx(L, i, x, y)] - feq[i]) / tau + Fi;
                int xt = wrap(x + ex_[i], L->nx);
                int yt = y + ey_[i];
                if (L->walls && (yt < 0 || yt >= L->ny)) {
                    double uw = (yt < 0) ? L->u_bottom : L->u_top;
                    double corr = -2.0 * w_[i] * 1.0 * (ex_[i] * uw) / cs2;
                    fnew[fidx(L, opp_[i], x, y)] = fpost + corr;
                } else {
                    yt = wrap(yt, L->ny);
                    fnew[fidx(L, i, xt, yt)] = fpost;
                }
            }
        }
    }
    orc_open_boundaries(L, fnew);   /* replaces what the periodic wrap carried across */
}

/* Fill populations with the equilibrium of given fields (rest state where NULL). */
void orc_init_equilibrium(const orc_lattice* L, const double* rho, const double* ux,
                          const double* uy, double* f) {
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t n = nidx(L, x, y);
            double feq[9];
            orc_feq(rho ? rho[n] : 1.0, ux ? ux[n] : 0.0, uy ? uy[n] : 0.0, feq);
            for (int i = 0; i < 9; i++) f[fidx(L, i, x, y)] = feq[i];
        }
}

/* ---------------------------------------------------------------------------------- */
/* Moving least squares transfer (Eq. 8-9, reading R5).                                 */
/* ---------------------------------------------------------------------------------- */

/* Solve the 3x3 system A Z = B for a 3 x m right-hand side (Gaussian elimination with
 * partial pivoting). A and B are overwritten. */
static void solve3(double A[3][3], double B[3][9], int m) {
    for (int c = 0; c < 3; c++) {
        int piv = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < 3; k++) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            for (int k = 0; k < m; k++) { double t = B[c][k]; B[c][k] = B[piv][k]; B[piv][k] = t; }
        }
        for (int r = c + 1; r < 3; r++) {
            double s = A[r][c] / A[c][c];
            for (int k = c; k < 3; k++) A[r][k] -= s * A[c][k];
            for (int k = 0; k < m; k++) B[r][k] -= s * B[c][k];
        }
    }
    for (int c = 2; c >= 0; c--) {
        for (int k = 0; k < m; k++) {
            double s = B[c][k];
            for (int j = c + 1; j < 3; j++) s -= A[c][j] * B[j][k];
            B[c][k] = s / A[c][c];
        }
    }
}

/*
 * Shape functions of the marker at (X, Y). The support is the 3x3 block of lattice
 * nodes centred on the node nearest to the marker (Fig. 1a). With weights
 * W_k = exp(-(r_k/alpha)^2), r_k = |x - x_k| / r_w, r_w = 2.6, alpha = 0.3 (Section 2.2),
 * minimising Eq. 9 over the coefficients a of the linear basis gives
 * a = A^-1 sum_k W_k p_k u_k with A = sum_k W_k p_k p_k^T. In the basis written about
 * the marker, U(X) = a_0, so phi_k = (A^-1 W_k p_k)_0 (Eq. 8), and the fitted slopes
 * a_1, a_2 give the gradient weights gx_k, gy_k.
 * Outputs lattice indices (ix[k], iy[k]); returns ORC_ERR_SUPPORT when a support node
 * falls outside the walls.
 */
int orc_mls(const orc_lattice* L, double X, double Y, int ix[9], int iy[9], double phi[9],
            double gx[9], double gy[9]) {
    const double rw = 2.6, alpha = 0.3;
    int cx = (int)floor(X + 0.5), cy = (int)floor(Y + 0.5);
    double A[3][3] = {{0}}, B[3][9];
    int status = ORC_OK;
    int k = 0;
    for (int b = -1; b <= 1; b++) {
        for (int a = -1; a <= 1; a++, k++) {
            int xk = cx + a, yk = cy + b;
            double dx = xk - X, dy = yk - Y;
            double r = sqrt(dx * dx + dy * dy) / rw;
            double Wk = exp(-(r / alpha) * (r / alpha));
            double p[3] = {1.0, dx, dy};
            for (int m = 0; m < 3; m++) {
                for (int n = 0; n < 3; n++) A[m][n] += Wk * p[m] * p[n];
                B[m][k] = Wk * p[m];
            }
            if (L->inflow) {   /* open channel: supports stay off the open columns (R26) */
                if (xk < 1 || xk > L->nx - 2) status = ORC_ERR_SUPPORT;
                ix[k] = xk < 0 ? 0 : (xk >= L->nx ? L->nx - 1 : xk);
            } else {
                ix[k] = wrap(xk, L->nx);
            }
            if (L->walls) {
                if (yk < 0 || yk >= L->ny) status = ORC_ERR_SUPPORT;
                iy[k] = yk < 0 ? 0 : (yk >= L->ny ? L->ny - 1 : yk);
            } else {
                iy[k] = wrap(yk, L->ny);
            }
        }
    }
    solve3(A, B, 9);
    for (k = 0; k < 9; k++) {
        phi[k] = B[0][k];
        if (gx) gx[k] = B[1][k];
        if (gy) gy[k] = B[2][k];
    }
    return status;
}

/*
 * Interpolate at (X, Y) (Eq. 8): out = {ux, uy, rho, p, dux/dx, dux/dy, duy/dx, duy/dy}.
 * The lattice velocity is Eq. 7 with the supplied force field fib (may be NULL).
 */
int orc_interp(const orc_lattice* L, const double* f, const double* fib, double X, double Y,
               double out[8]) {
    int ix[9], iy[9];
    double phi[9], gx[9], gy[9];
    int st = orc_mls(L, X, Y, ix, iy, phi, gx, gy);
    for (int m = 0; m < 8; m++) out[m] = 0.0;
    for (int k = 0; k < 9; k++) {
        double rho, ux, uy;
        node_macros(L, f, fib, ix[k], iy[k], &rho, &ux, &uy);
        out[0] += phi[k] * ux;
        out[1] += phi[k] * uy;
        out[2] += phi[k] * rho;
        out[3] += phi[k] * rho / 3.0;
        out[4] += gx[k] * ux;
        out[5] += gy[k] * ux;
        out[6] += gx[k] * uy;
        out[7] += gy[k] * uy;
    }
    return st;
}

/* Interpolate an arbitrary nodal scalar field v (nx*ny) at (X, Y) with Eq. 8. */
int orc_interp_scalar(const orc_lattice* L, const double* v, double X, double Y, double* out) {
    int ix[9], iy[9];
    double phi[9];
    int st = orc_mls(L, X, Y, ix, iy, phi, NULL, NULL);
    double s = 0.0;
    for (int k = 0; k < 9; k++) s += phi[k] * v[nidx(L, ix[k], iy[k])];
    *out = s;
    return st;
}

/* Spreading (step 3 / step iii): f_ib(x_k) += c phi_k F at the marker's support. */
int orc_spread(const orc_lattice* L, double X, double Y, double Fx, double Fy, double c,
               double* fib) {
    int ix[9], iy[9];
    double phi[9];
    int st = orc_mls(L, X, Y, ix, iy, phi, NULL, NULL);
    size_t N = (size_t)L->nx * (size_t)L->ny;
    for (int k = 0; k < 9; k++) {
        size_t n = nidx(L, ix[k], iy[k]);
        fib[n] += c * phi[k] * Fx;
        fib[N + n] += c * phi[k] * Fy;
    }
    return st;
}

/* ---------------------------------------------------------------------------------- */
/* Membrane mechanics (Section 2.2.1, Eq. 10-14).                                       */
/* Ring of n vertices, counter-clockwise; element l joins vertex l to vertex l+1.       */
/* ---------------------------------------------------------------------------------- */

/* Signed turning angle at vertex v between incoming edge a and outgoing edge b (R6). */
static double turning_angle(const double* xy, int n, int v) {
    int vl = (v + n - 1) % n, vr = (v + 1) % n;
    double ax = xy[2 * v] - xy[2 * vl], ay = xy[2 * v + 1] - xy[2 * vl + 1];
    double bx = xy[2 * vr] - xy[2 * v], by = xy[2 * vr + 1] - xy[2 * v + 1];
    return atan2(ax * by - ay * bx, ax * bx + ay * by);
}

/* Enclosed area by Green's theorem with the factor 1/2 (reading R7). */
double orc_area(const double* xy, int n) {
    double s = 0.0;
    for (int l = 0; l < n; l++) {
        int r = (l + 1) % n;
        s += xy[2 * l] * xy[2 * r + 1] - xy[2 * r] * xy[2 * l + 1];
    }
    return 0.5 * s;
}

double orc_perimeter(const double* xy, int n) {
    double s = 0.0;
    for (int l = 0; l < n; l++) {
        int r = (l + 1) % n;
        s += hypot(xy[2 * r] - xy[2 * l], xy[2 * r + 1] - xy[2 * l + 1]);
    }
    return s;
}

/* Stress-free reference: element lengths L0[l], vertex angles th0[v], area A0. */
void orc_membrane_reference(const double* xy, int n, double* L0, double* th0, double* A0) {
    for (int l = 0; l < n; l++) {
        int r = (l + 1) % n;
        L0[l] = hypot(xy[2 * r] - xy[2 * l], xy[2 * r + 1] - xy[2 * l + 1]);
    }
    for (int v = 0; v < n; v++) th0[v] = turning_angle(xy, n, v);
    *A0 = orc_area(xy, n);
}

/* Total elastic energy: Eq. 10 (stretch), the bending energy of reading R6, and the
 * area energy whose gradient is Eq. 14, k_a p_ref A0/2 (1 - A/A0)^2 with p_ref = 1/3. */
double orc_membrane_energy(const double* xy, int n, const double* L0, const double* th0, double A0,
                           double ks, double kb, double ka) {
    double E = 0.0;
    for (int l = 0; l < n; l++) {
        int r = (l + 1) % n;
        double len = hypot(xy[2 * r] - xy[2 * l], xy[2 * r + 1] - xy[2 * l + 1]);
        E += 0.5 * ks * (len - L0[l]) * (len - L0[l]);
    }
    for (int v = 0; v < n; v++) E += kb * (1.0 - cos(turning_angle(xy, n, v) - th0[v]));
    double A = orc_area(xy, n);
    E += ka * (1.0 / 3.0) * 0.5 * A0 * (1.0 - A / A0) * (1.0 - A / A0);
    return E;
}

/* Internal nodal forces F^int = F^s + F^b + F^a (Eq. 11, 13 as read in R6, 14). */
void orc_membrane_force(const double* xy, int n, const double* L0, const double* th0, double A0,
                        double ks, double kb, double ka, double* F) {
    for (int m = 0; m < 2 * n; m++) F[m] = 0.0;
    /* Eq. 11: stretch of element l between v1 = l and v2 = l + 1 */
    for (int l = 0; l < n; l++) {
        int v1 = l, v2 = (l + 1) % n;
        double r12x = xy[2 * v1] - xy[2 * v2], r12y = xy[2 * v1 + 1] - xy[2 * v2 + 1];
        double len = hypot(r12x, r12y);
        double s = -ks * (len - L0[l]) / len;
        F[2 * v1] += s * r12x;
        F[2 * v1 + 1] += s * r12y;
        F[2 * v2] -= s * r12x;
        F[2 * v2 + 1] -= s * r12y;
    }
    /* Eq. 13 (R6): F = -k_b sin(theta - theta_0) d(theta)/dX at v_left, v, v_right */
    for (int v = 0; v < n; v++) {
        int vl = (v + n - 1) % n, vr = (v + 1) % n;
        double ax = xy[2 * v] - xy[2 * vl], ay = xy[2 * v + 1] - xy[2 * vl + 1];
        double bx = xy[2 * vr] - xy[2 * v], by = xy[2 * vr + 1] - xy[2 * v + 1];
        double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
        double th = atan2(ax * by - ay * bx, ax * bx + ay * by);
        double s = kb * sin(th - th0[v]);
        /* d(theta)/dX_left = (-a_y, a_x)/|a|^2, d(theta)/dX_right = (-b_y, b_x)/|b|^2 */
        double dlx = -ay / a2, dly = ax / a2;
        double drx = -by / b2, dry = bx / b2;
        F[2 * vl] -= s * dlx;
        F[2 * vl + 1] -= s * dly;
        F[2 * vr] -= s * drx;
        F[2 * vr + 1] -= s * dry;
        F[2 * v] += s * (dlx + drx);
        F[2 * v + 1] += s * (dly + dry);
    }
    /* Eq. 14: F^a_l = -k_a (1 - A/A0) p_ref n^-_l l_l, half to each end node (R7) */
    double A = orc_area(xy, n);
    double pref = 1.0 / 3.0;
    for (int l = 0; l < n; l++) {
        int v1 = l, v2 = (l + 1) % n;
        double dx = xy[2 * v2] - xy[2 * v1], dy = xy[2 * v2 + 1] - xy[2 * v1 + 1];
        /* n^- l = -(dy, -dx) */
        double nmx = -dy, nmy = dx;
        double Fx = -ka * (1.0 - A / A0) * pref * nmx;
        double Fy = -ka * (1.0 - A / A0) * pref * nmy;
        F[2 * v1] += 0.5 * Fx;
        F[2 * v1 + 1] += 0.5 * Fy;
        F[2 * v2] += 0.5 * Fx;
        F[2 * v2 + 1] += 0.5 * Fy;
    }
}

/* ---------------------------------------------------------------------------------- */
/* Observables (Section 3.1, 3.2).                                                      */
/* out = {area, perimeter, D, xc, yc, Sw, inclination, I_max}; D from the eigenvalues   */
/* of the area second-moment tensor (R15); inclination of the major axis in radians.    */
/* ---------------------------------------------------------------------------------- */
void orc_observables(const double* xy, int n, double out[8]) {
    /* coordinates relative to the first vertex (translation-invariant quantities) */
    double x0 = xy[0], y0 = xy[1];
    double A2 = 0.0, sx = 0.0, sy = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int i = 0; i < n; i++) {
        int j = (i + 1) % n;
        double xi = xy[2 * i] - x0, yi = xy[2 * i + 1] - y0;
        double xj = xy[2 * j] - x0, yj = xy[2 * j + 1] - y0;
        double c = xi * yj - xj * yi;
        A2 += c;
        sx += (xi + xj) * c;
        sy += (yi + yj) * c;
        sxx += (xi * xi + xi * xj + xj * xj) * c;
        syy += (yi * yi + yi * yj + yj * yj) * c;
        sxy += (xi * yj + 2.0 * xi * yi + 2.0 * xj * yj + xj * yi) * c;
    }
    double A = 0.5 * A2;
    double cx = sx / (6.0 * A), cy = sy / (6.0 * A);
    double Ixx = sxx / 12.0 - A * cx * cx;
    double Iyy = syy / 12.0 - A * cy * cy;
    double Ixy = sxy / 24.0 - A * cx * cy;
    double m = 0.5 * (Ixx + Iyy);
    double d = sqrt(0.25 * (Ixx - Iyy) * (Ixx - Iyy) + Ixy * Ixy);
    double lmax = (m + d) / A, lmin = (m - d) / A;
    double a = 2.0 * sqrt(lmax), b = 2.0 * sqrt(lmin > 0.0 ? lmin : 0.0);
    double P = orc_perimeter(xy, n);
    out[0] = A;
    out[1] = P;
    out[2] = (a - b) / (a + b);
    out[3] = cx + x0;
    out[4] = cy + y0;
    out[5] = A / (P * P / (4.0 * M_PI));
    out[6] = 0.5 * atan2(2.0 * Ixy, Ixx - Iyy);
    out[7] = lmax;
}

/* ---------------------------------------------------------------------------------- */
/* Node integrators.                                                                    */
/* ---------------------------------------------------------------------------------- */

/* Eq. 25 (Kinematic): x^{n+1} = 2/3 (2 x^n - x^{n-1}/2 + xdot); forward Euler if first. */
void orc_kinematic_advance(int n2, const double* X, const double* Xm1, const double* xdot,
                           int first, double* Xnew) {
    for (int m = 0; m < n2; m++)
        Xnew[m] = first ? X[m] + xdot[m]
                        : (2.0 / 3.0) * (2.0 * X[m] - 0.5 * Xm1[m] + xdot[m]);
}

/* Eq. 23 (Verlet with the interpolated tentative velocity) and Eq. 24 (velocity). */
void orc_dynamic_advance(int n2, const double* X, const double* Xm1, const double* xdot0,
                         const double* Ftot, double m, double* Xnew, double* uv) {
    for (int k = 0; k < n2; k++) {
        Xnew[k] = X[k] + xdot0[k] + 0.5 * Ftot[k] / m;
        uv[k] = 1.5 * Xnew[k] - 2.0 * X[k] + 0.5 * Xm1[k];
    }
}

/* ---------------------------------------------------------------------------------- */
/* Capsule-capsule repulsion (Section 3.4, Eq. 27; readings R23, R24).                   */
/* ---------------------------------------------------------------------------------- */
/* Outward unit normal at vertex v of a counter-clockwise ring of n vertices: the
 * normalised sum of the outward normals (dy, -dx)/l of elements v-1 and v. */
void orc_vertex_normal(const double* X, int n, int v, double out[2]) {
    int vl = (v + n - 1) % n, vr = (v + 1) % n;
    double ax = X[2 * v] - X[2 * vl], ay = X[2 * v + 1] - X[2 * vl + 1];
    double bx = X[2 * vr] - X[2 * v], by = X[2 * vr + 1] - X[2 * v + 1];
    double la = hypot(ax, ay), lb = hypot(bx, by);
    double nx = ay / la + by / lb, ny = -ax / la - bx / lb;
    double ln = hypot(nx, ny);
    out[0] = nx / ln;
    out[1] = ny / ln;
}

/* Minimum-image difference a - b along an axis of period P (P = 0: not periodic). */
static double min_image(double d, double P) {
    if (P > 0.0) d -= P * floor(d / P + 0.5);
    return d;
}

/* F[c] (2 n_c doubles each, overwritten): on every vertex 1 of ring c, from every vertex
 * 2 of every other ring at distance d < rc, coeff * sqrt(dx / d^5) along the inward
 * normal at vertex 1 (Eq. 27 with coeff = 1e-4 / (8 sqrt 2) and dx = 1 lattice unit).
 * Periods px, py (0: none) for minimum-image distances. */
void orc_repulsion(const double* const* X, const int* n, int ncaps, double rc, double coeff, double px,
                   double py, double* const* F) {
    for (int a = 0; a < ncaps; a++) {
        for (int v = 0; v < n[a]; v++) {
            double nrm[2];
            orc_vertex_normal(X[a], n[a], v, nrm);
            double f = 0.0;
            for (int b = 0; b < ncaps; b++) {
                if (b == a) continue;
                for (int w = 0; w < n[b]; w++) {
                    double dx = min_image(X[a][2 * v] - X[b][2 * w], px);
                    double dy = min_image(X[a][2 * v + 1] - X[b][2 * w + 1], py);
                    double d = sqrt(dx * dx + dy * dy);
                    if (d < rc) f += coeff * sqrt(1.0 / (d * d * d * d * d));
                }
            }
            F[a][2 * v] = -f * nrm[0];
            F[a][2 * v + 1] = -f * nrm[1];
        }
    }
}


/* ---------------------------------------------------------------------------------- */
/* Simulation: lattice + capsules, stepped with the Kinematic (Section 2.4, steps i-viii)*/
/* or Dynamic (Section 2.3, steps 1-8) scheme.                                          */
/* ---------------------------------------------------------------------------------- */
typedef struct {
    int n;
    double ks, kb, ka, m;
    double *X, *Xm1, *uv, *Fint, *Fext, *Fpp, *L0, *th0;
    double A0, P0;
    int age;
    /* rigid particle (R27-R30): body state {c_x, c_y, theta, u_x, u_y, omega} at n and
     * at n - 1, mass, moment of inertia, reference offsets r_v, last load {F_x, F_y, M} */
    int rigid;
    double body[6], prev[6], mass, inertia, load[3];
    double* R0;
} orc_capsule;

typedef struct {
    orc_lattice L;
    double *f, *fnew, *fib, *fibnew;
    int ncaps, cap_capacity;
    orc_capsule* caps;
    long long step;
    int status;
    double rep_rc, rep_c;   /* repulsion cut-off (0: off) and coefficient of Eq. 27 */
} orc_sim;

/* Repulsion forces of all capsules of a simulation at their current positions. */
static void sim_repulsion(orc_sim* s) {
    if (s->rep_rc <= 0.0 || s->ncaps < 2) {
        for (int c = 0; c < s->ncaps; c++) memset(s->caps[c].Fpp, 0, 2 * s->caps[c].n * sizeof(double));
        return;
    }
    const double** X = (const double**)malloc(s->ncaps * sizeof(double*));
    int* n = (int*)malloc(s->ncaps * sizeof(int));
    double** F = (double**)malloc(s->ncaps * sizeof(double*));
    for (int c = 0; c < s->ncaps; c++) {
        X[c] = s->caps[c].X;
        n[c] = s->caps[c].n;
        F[c] = s->caps[c].Fpp;
    }
    orc_repulsion(X, n, s->ncaps, s->rep_rc, s->rep_c, s->L.inflow ? 0.0 : (double)s->L.nx,
                  s->L.walls ? 0.0 : (double)s->L.ny, F);
    free(X);
    free(n);
    free(F);
}

void orc_sim_set_repulsion(orc_sim* s, double rc, double coeff) {
    s->rep_rc = rc;
    s->rep_c = coeff;
}

orc_sim* orc_sim_create(const orc_lattice* L) {
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->L = *L;
    size_t N = (size_t)L->nx * (size_t)L->ny;
    s->f = (double*)calloc(9 * N, sizeof(double));
    s->fnew = (double*)calloc(9 * N, sizeof(double));
    s->fib = (double*)calloc(2 * N, sizeof(double));
    s->fibnew = (double*)calloc(2 * N, sizeof(double));
    orc_init_equilibrium(L, NULL, NULL, NULL, s->f);
    return s;
}

void orc_sim_destroy(orc_sim* s) {
    if (!s) return;
    for (int c = 0; c < s->ncaps; c++) {
        orc_capsule* k = &s->caps[c];
        free(k->X); free(k->Xm1); free(k->uv); free(k->Fint); free(k->Fext); free(k->Fpp);
        free(k->L0); free(k->th0); free(k->R0);
    }
    free(s->caps);
    free(s->f); free(s->fnew); free(s->fib); free(s->fibnew);
    free(s);
}

void orc_sim_init_fields(orc_sim* s, const double* rho, const double* ux, const double* uy) {
    orc_init_equilibrium(&s->L, rho, ux, uy, s->f);
    orc_open_boundaries(&s->L, s->f);   /* the open columns hold their prescribed state */
}

/* direct access for tests: populations (9*N, pre-collision) and last spread force */
double* orc_sim_populations(orc_sim* s) { return s->f; }
double* orc_sim_force_field(orc_sim* s) { return s->fib; }

int orc_sim_add_capsule(orc_sim* s, const double* xy, int n, double ks, double kb, double ka,
                        double m) {
    if (s->ncaps == s->cap_capacity) {
        s->cap_capacity = s->cap_capacity ? 2 * s->cap_capacity : 8;
        s->caps = (orc_capsule*)realloc(s->caps, (size_t)s->cap_capacity * sizeof(orc_capsule));
    }
    orc_capsule* k = &s->caps[s->ncaps];
    memset(k, 0, sizeof(*k));
    k->n = n; k->ks = ks; k->kb = kb; k->ka = ka; k->m = m;
    k->X = (double*)malloc(2 * n * sizeof(double));
    k->Xm1 = (double*)malloc(2 * n * sizeof(double));
    k->uv = (double*)calloc(2 * n, sizeof(double));
    k->Fint = (double*)calloc(2 * n, sizeof(double));
    k->Fext = (double*)calloc(2 * n, sizeof(double));
    k->Fpp = (double*)calloc(2 * n, sizeof(double));
    k->L0 = (double*)malloc(n * sizeof(double));
    k->th0 = (double*)malloc(n * sizeof(double));
    memcpy(k->X, xy, 2 * n * sizeof(double));
    memcpy(k->Xm1, xy, 2 * n * sizeof(double));
    orc_membrane_reference(xy, n, k->L0, k->th0, &k->A0);
    k->P0 = orc_perimeter(xy, n);
    return s->ncaps++;
}

/* Markers of a rigid ring from its body state: X_v = c + R(theta) r_v; velocities
 * u + omega x (X_v - c). */
static void rigid_markers(orc_capsule* k) {
    const double c = cos(k->body[2]), sn = sin(k->body[2]);
    for (int v = 0; v < k->n; v++) {
        double rx = c * k->R0[2 * v] - sn * k->R0[2 * v + 1];
        double ry = sn * k->R0[2 * v] + c * k->R0[2 * v + 1];
        k->X[2 * v] = k->body[0] + rx;
        k->X[2 * v + 1] = k->body[1] + ry;
        k->uv[2 * v] = k->body[3] - k->body[5] * ry;
        k->uv[2 * v + 1] = k->body[4] + k->body[5] * rx;
    }
}

/* Add a rigid particle (R27): ring xy (counter-clockwise), mass and moment of inertia
 * about its area centroid; at rest. Returns its id. */
int orc_sim_add_rigid(orc_sim* s, const double* xy, int n, double mass, double inertia) {
    const int id = orc_sim_add_capsule(s, xy, n, 0.0, 0.0, 0.0, mass / n);
    orc_capsule* k = &s->caps[id];
    double o[8];
    orc_observables(xy, n, o);   /* area centroid in o[3], o[4] */
    k->rigid = 1;
    k->mass = mass;
    k->inertia = inertia;
    k->R0 = (double*)malloc(2 * n * sizeof(double));
    for (int v = 0; v < n; v++) {
        k->R0[2 * v] = xy[2 * v] - o[3];
        k->R0[2 * v + 1] = xy[2 * v + 1] - o[4];
    }
    for (int a = 0; a < 6; a++) k->body[a] = k->prev[a] = 0.0;
    k->body[0] = k->prev[0] = o[3];
    k->body[1] = k->prev[1] = o[4];
    rigid_markers(k);
    return id;
}

/* Body state of rigid particle id: {c_x, c_y, theta, u_x, u_y, omega, F_x, F_y, M} (the
 * last load). Returns 1 if id is not a rigid particle. */
int orc_sim_read_rigid(orc_sim* s, int id, double out[9]) {
    if (id < 0 || id >= s->ncaps || !s->caps[id].rigid) return 1;
    orc_capsule* k = &s->caps[id];
    for (int a = 0; a < 6; a++) out[a] = k->body[a];
    for (int a = 0; a < 3; a++) out[6 + a] = k->load[a];
    return 0;
}

/* Start a capsule from positions other than its stress-free shape (X^n = X^{n-1} = xy). */
int orc_sim_set_capsule_positions(orc_sim* s, int id, const double* xy) {
    if (id < 0 || id >= s->ncaps || s->caps[id].rigid) return 1;
    orc_capsule* k = &s->caps[id];
    memcpy(k->X, xy, 2 * k->n * sizeof(double));
    memcpy(k->Xm1, xy, 2 * k->n * sizeof(double));
    k->age = 0;
    return 0;
}

static void swap_ptr(double** a, double** b) { double* t = *a; *a = *b; *b = t; }

/* Kinematic IB, steps i-viii (Section 2.4). */
static void kinematic_step(orc_sim* s) {
    orc_lattice* L = &s->L;
    size_t N = (size_t)L->nx * (size_t)L->ny;
    memset(s->fibnew, 0, 2 * N * sizeof(double));
    /* i: internal forces at X^n (and the capsule-capsule repulsion of Eq. 27);
     * ii-iii: spread with c_v = 1 */
    sim_repulsion(s);
    for (int c = 0; c < s->ncaps; c++) {
        orc_capsule* k = &s->caps[c];
        orc_membrane_force(k->X, k->n, k->L0, k->th0, k->A0, k->ks, k->kb, k->ka, k->Fint);
        for (int v = 0; v < k->n; v++) {
            k->Fext[2 * v] = k->Fext[2 * v + 1] = 0.0;
            if (orc_spread(L, k->X[2 * v], k->X[2 * v + 1], k->Fint[2 * v] + k->Fpp[2 * v],
                           k->Fint[2 * v + 1] + k->Fpp[2 * v + 1], 1.0, s->fibnew))
                s->status = ORC_ERR_SUPPORT;
        }
    }
    /* iv-v: forcing term and lattice update */
    orc_collide_stream(L, s->f, s->fibnew, s->fnew);
    swap_ptr(&s->f, &s->fnew);
    swap_ptr(&s->fib, &s->fibnew);
    /* vi-viii: interpolate the updated velocity (with half the spread force) at X^n
     * and advance with Eq. 25 */
    for (int c = 0; c < s->ncaps; c++) {
        orc_capsule* k = &s->caps[c];
        double* xdot = (double*)malloc(2 * k->n * sizeof(double));
        double* Xnew = (double*)malloc(2 * k->n * sizeof(double));
        for (int v = 0; v < k->n; v++) {
            double o[8];
            if (orc_interp(L, s->f, s->fib, k->X[2 * v], k->X[2 * v + 1], o))
                s->status = ORC_ERR_SUPPORT;
            xdot[2 * v] = o[0];
            xdot[2 * v + 1] = o[1];
        }
        orc_kinematic_advance(2 * k->n, k->X, k->Xm1, xdot, k->age == 0, Xnew);
        memcpy(k->Xm1, k->X, 2 * k->n * sizeof(double));
        memcpy(k->X, Xnew, 2 * k->n * sizeof(double));
        memcpy(k->uv, xdot, 2 * k->n * sizeof(double));
        k->age++;
        free(xdot);
        free(Xnew);
    }
}

/* Hydrodynamic traction on the elements of a ring of n vertices (Eq. 15-16, reading
 * R12): probes at the element centroid +/- 1.2 n+; each element's force goes half to
 * each of its two vertices, accumulated into Fext[2n]. */
int orc_tractions(const orc_lattice* L, const double* f, const double* fib, const double* X,
                  int n, double* Fext) {
    int st = ORC_OK;
    double nu = (L->tau - 0.5) / 3.0;
    for (int m = 0; m < 2 * n; m++) Fext[m] = 0.0;
    for (int l = 0; l < n; l++) {
        int v1 = l, v2 = (l + 1) % n;
        double dx = X[2 * v2] - X[2 * v1], dy = X[2 * v2 + 1] - X[2 * v1 + 1];
        double len = hypot(dx, dy);
        double npx = dy / len, npy = -dx / len; /* outward normal, CCW ring (R7) */
        double cx = 0.5 * (X[2 * v1] + X[2 * v2]);
        double cy = 0.5 * (X[2 * v1 + 1] + X[2 * v2 + 1]);
        double op[8], om[8];
        if (orc_interp(L, f, fib, cx + 1.2 * npx, cy + 1.2 * npy, op)) st = ORC_ERR_SUPPORT;
        if (orc_interp(L, f, fib, cx - 1.2 * npx, cy - 1.2 * npy, om)) st = ORC_ERR_SUPPORT;
        /* viscous stress tau = rho nu (grad u + grad u^T) at each probe */
        double tp[2][2], tm[2][2];
        double gp[2][2] = {{op[4], op[5]}, {op[6], op[7]}};
        double gm[2][2] = {{om[4], om[5]}, {om[6], om[7]}};
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                tp[a][b] = op[2] * nu * (gp[a][b] + gp[b][a]);
                tm[a][b] = om[2] * nu * (gm[a][b] + gm[b][a]);
            }
        /* Eq. 15 */
        double Fpx = -(op[3] - om[3]) * npx * len;
        double Fpy = -(op[3] - om[3]) * npy * len;
        /* Eq. 16 */
        double Ftx = ((tp[0][0] - tm[0][0]) * npx + (tp[0][1] - tm[0][1]) * npy) * len;
        double Fty = ((tp[1][0] - tm[1][0]) * npx + (tp[1][1] - tm[1][1]) * npy) * len;
        Fext[2 * v1] += 0.5 * (Fpx + Ftx);
        Fext[2 * v1 + 1] += 0.5 * (Fpy + Fty);
        Fext[2 * v2] += 0.5 * (Fpx + Ftx);
        Fext[2 * v2 + 1] += 0.5 * (Fpy + Fty);
    }
    return st;
}

/* Fluid load on a rigid ring of n vertices about c (Eq. 17-18, reading R28): for every
 * element the outer probe's traction (tau+ . n+ - p+ n+) l_l, summed (F_x, F_y) and its
 * moment (r_l x f_l) about c, into load[3]. fext (may be NULL) gets half of each
 * element's force at each end vertex. */
int orc_rigid_load(const orc_lattice* L, const double* f, const double* fib, const double* X, int n,
                   double cx, double cy, double load[3], double* fext) {
    int st = ORC_OK;
    double nu = (L->tau - 0.5) / 3.0;
    load[0] = load[1] = load[2] = 0.0;
    if (fext) for (int m = 0; m < 2 * n; m++) fext[m] = 0.0;
    for (int l = 0; l < n; l++) {
        int v1 = l, v2 = (l + 1) % n;
        double dx = X[2 * v2] - X[2 * v1], dy = X[2 * v2 + 1] - X[2 * v1 + 1];
        double len = hypot(dx, dy);
        double npx = dy / len, npy = -dx / len;   /* outward normal (R7) */
        double mx = 0.5 * (X[2 * v1] + X[2 * v2]), my = 0.5 * (X[2 * v1 + 1] + X[2 * v2 + 1]);
        double op[8];
        if (orc_interp(L, f, fib, mx + 1.2 * npx, my + 1.2 * npy, op)) st = ORC_ERR_SUPPORT;
        double g[2][2] = {{op[4], op[5]}, {op[6], op[7]}}, t[2][2];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) t[a][b] = op[2] * nu * (g[a][b] + g[b][a]);
        /* Eq. 17 term of element l */
        double fx = (t[0][0] * npx + t[0][1] * npy - op[3] * npx) * len;
        double fy = (t[1][0] * npx + t[1][1] * npy - op[3] * npy) * len;
        load[0] += fx;
        load[1] += fy;
        /* Eq. 18 term: r_l x f_l, r_l from c to the element centroid */
        load[2] += (mx - cx) * fy - (my - cy) * fx;
        if (fext) {
            fext[2 * v1] += 0.5 * fx; fext[2 * v1 + 1] += 0.5 * fy;
            fext[2 * v2] += 0.5 * fx; fext[2 * v2 + 1] += 0.5 * fy;
        }
    }
    return st;
}

/* One rigid-body update (Eq. 19-20, reading R29). body = {c_x, c_y, theta, u_x, u_y,
 * omega} at n, prev the same at n - 1; acceleration from load = {F_x, F_y, M} over mass
 * and inertia. On return body holds n + 1 and prev n. */
void orc_rigid_advance(double body[6], double prev[6], const double load[3], double mass, double inertia) {
    const double acc[3] = {load[0] / mass, load[1] / mass, load[2] / inertia};
    double next[6];
    for (int a = 0; a < 3; a++) {
        /* Eq. 19 (a = 0, 1) and Eq. 20 (a = 2) */
        next[3 + a] = (2.0 / 3.0) * (2.0 * body[3 + a] - 0.5 * prev[3 + a] + acc[a]);
        /* position and angle: the same backward form (R29) */
        next[a] = (2.0 / 3.0) * (2.0 * body[a] - 0.5 * prev[a] + next[3 + a]);
    }
    for (int a = 0; a < 6; a++) {
        prev[a] = body[a];
        body[a] = next[a];
    }
}

/* Dynamic IB, steps 1-8 (Section 2.3.2). */
static void dynamic_step(orc_sim* s) {
    orc_lattice* L = &s->L;
    size_t N = (size_t)L->nx * (size_t)L->ny;
    memset(s->fibnew, 0, 2 * N * sizeof(double));
    sim_repulsion(s);   /* Eq. 27 at X^n, part of the total force of step 7 */
    /* 1-3: U = I(u^n) of the populations before any IB force (R1d), F_l = (U_b - U)/dt,
     * spread. U is also the tentative velocity of step 8 (R11). */
    double** Ucap = (double**)malloc((s->ncaps > 0 ? s->ncaps : 1) * sizeof(double*));
    for (int c = 0; c < s->ncaps; c++) {
        orc_capsule* k = &s->caps[c];
        int n = k->n;
        double* F = (double*)malloc(2 * n * sizeof(double));
        double* U = (double*)malloc(2 * n * sizeof(double));
        Ucap[c] = U;
        for (int v = 0; v < n; v++) {
            double o[8];
            if (orc_interp(L, s->f, NULL, k->X[2 * v], k->X[2 * v + 1], o))
                s->status = ORC_ERR_SUPPORT;
            U[2 * v] = o[0];
            U[2 * v + 1] = o[1];
            if (k->rigid) {
                /* desired velocity: the rigid-body motion (R27) */
                k->uv[2 * v] = k->body[3] - k->body[5] * (k->X[2 * v + 1] - k->body[1]);
                k->uv[2 * v + 1] = k->body[4] + k->body[5] * (k->X[2 * v] - k->body[0]);
            } else if (k->age == 0) {
                /* start-up: node velocity = fluid velocity, X^{-1} = X^0 - u_v^0 */
                k->uv[2 * v] = o[0];
                k->uv[2 * v + 1] = o[1];
                k->Xm1[2 * v] = k->X[2 * v] - o[0];
                k->Xm1[2 * v + 1] = k->X[2 * v + 1] - o[1];
            }
            F[2 * v] = k->uv[2 * v] - o[0];
            F[2 * v + 1] = k->uv[2 * v + 1] - o[1];
        }
        for (int v = 0; v < n; v++) {
            int vl = (v + n - 1) % n, vr = (v + 1) % n;
            double ll = hypot(k->X[2 * v] - k->X[2 * vl], k->X[2 * v + 1] - k->X[2 * vl + 1]);
            double lr = hypot(k->X[2 * vr] - k->X[2 * v], k->X[2 * vr + 1] - k->X[2 * v + 1]);
            double cl = 1.0 * 0.5 * (ll + lr); /* reading R4 */
            if (orc_spread(L, k->X[2 * v], k->X[2 * v + 1], F[2 * v], F[2 * v + 1], cl, s->fibnew))
                s->status = ORC_ERR_SUPPORT;
        }
        free(F);
    }
    /* 4-6: forcing term, lattice update, macroscopic quantities */
    orc_collide_stream(L, s->f, s->fibnew, s->fnew);
    swap_ptr(&s->f, &s->fnew);
    swap_ptr(&s->fib, &s->fibnew);
    /* 7-8: total force and Verlet update (rigid particles: Eq. 17-20) */
    for (int c = 0; c < s->ncaps; c++) {
        orc_capsule* k = &s->caps[c];
        int n = k->n;
        if (k->rigid) {
            if (orc_rigid_load(L, s->f, NULL, k->X, n, k->body[0], k->body[1], k->load, k->Fext))
                s->status = ORC_ERR_SUPPORT;
            for (int v = 0; v < n; v++) {   /* Eq. 27 on the markers (R28) */
                k->load[0] += k->Fpp[2 * v];
                k->load[1] += k->Fpp[2 * v + 1];
                k->load[2] += (k->X[2 * v] - k->body[0]) * k->Fpp[2 * v + 1] -
                              (k->X[2 * v + 1] - k->body[1]) * k->Fpp[2 * v];
            }
            orc_rigid_advance(k->body, k->prev, k->load, k->mass, k->inertia);
            memcpy(k->Xm1, k->X, 2 * n * sizeof(double));
            rigid_markers(k);
            k->age++;
            continue;
        }
        double* Ftot = (double*)malloc(2 * n * sizeof(double));
        double* Xnew = (double*)malloc(2 * n * sizeof(double));
        /* 7: probe tractions on the updated populations (R1d), internal forces at X^n */
        if (orc_tractions(L, s->f, NULL, k->X, n, k->Fext)) s->status = ORC_ERR_SUPPORT;
        orc_membrane_force(k->X, n, k->L0, k->th0, k->A0, k->ks, k->kb, k->ka, k->Fint);
        for (int m = 0; m < 2 * n; m++) Ftot[m] = k->Fint[m] + k->Fext[m] + k->Fpp[m];
        /* 8: Eq. 23 with the tentative velocity U of step 1 (R11), Eq. 24 */
        orc_dynamic_advance(2 * n, k->X, k->Xm1, Ucap[c], Ftot, k->m, Xnew, k->uv);
        memcpy(k->Xm1, k->X, 2 * n * sizeof(double));
        memcpy(k->X, Xnew, 2 * n * sizeof(double));
        k->age++;
        free(Ftot);
        free(Xnew);
    }
    for (int c = 0; c < s->ncaps; c++) free(Ucap[c]);
    free(Ucap);
}

/* scheme: 0 = Kinematic, 1 = Dynamic. Returns the sticky status. */
int orc_sim_step(orc_sim* s, long long nsteps, int scheme) {
    if (scheme == 0)
        for (int c = 0; c < s->ncaps; c++)
            if (s->caps[c].rigid) return ORC_ERR_STATE;   /* R30 */
    for (long long t = 0; t < nsteps; t++) {
        if (scheme == 0) kinematic_step(s);
        else dynamic_step(s);
        s->step++;
    }
    return s->status;
}

/* Fields at the current time: rho and u of Eq. 6-7 with half of g + last spread force. */
void orc_sim_read_fields(orc_sim* s, double* rho, double* ux, double* uy) {
    orc_macros(&s->L, s->f, s->fib, rho, ux, uy);
}

/* Capsule state: positions X^n, node velocities (Kinematic: the last interpolated
 * velocity; Dynamic: u_v of Eq. 24), last internal and external nodal forces. */
int orc_sim_read_capsule(orc_sim* s, int id, double* xy, double* vel, double* fint, double* fext) {
    if (id < 0 || id >= s->ncaps) return 1;
    orc_capsule* k = &s->caps[id];
    if (xy) memcpy(xy, k->X, 2 * k->n * sizeof(double));
    if (vel) memcpy(vel, k->uv, 2 * k->n * sizeof(double));
    if (fint) memcpy(fint, k->Fint, 2 * k->n * sizeof(double));
    if (fext) memcpy(fext, k->Fext, 2 * k->n * sizeof(double));
    return 0;
}

/* Last repulsion forces of capsule id (2n doubles). */
int orc_sim_read_repulsion(orc_sim* s, int id, double* fpp) {
    if (id < 0 || id >= s->ncaps) return 1;
    memcpy(fpp, s->caps[id].Fpp, 2 * s->caps[id].n * sizeof(double));
    return 0;
}

/* out = {area, perimeter, D, xc, yc, Sw, inclination, delta_p} */
int orc_sim_observables(orc_sim* s, int id, double out[8]) {
    if (id < 0 || id >= s->ncaps) return 1;
    orc_capsule* k = &s->caps[id];
    double o[8];
    orc_observables(k->X, k->n, o);
    for (int m = 0; m < 7; m++) out[m] = o[m];
    out[7] = (o[1] - k->P0) / k->P0;
    return 0;
}

long long orc_sim_step_count(orc_sim* s) { return s->step; }
