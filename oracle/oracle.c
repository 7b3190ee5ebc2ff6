/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the IB-LB wetting time step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the CPU
 * baseline of bench.py; never by the product path.  It shares no code with
 * the CUDA library.  Every function follows one passage of the paper
 * (Bellantoni et al., arXiv 2503.20605), cited in its comment; where the
 * paper is silent the reading taken is stated in the comment ("Reading").
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared oracle.c -lm
 * (-fopenmp is optional: it only shares the independent cells of the
 *  stream-collide loop among threads; the results are the same bits.)
 * (-ffp-contract=off keeps every product and sum individually rounded, so that
 *  the decisions taken in floating point -- in/out of a cell -- are those of
 *  plain IEEE arithmetic.)
 *
 * Parity: all functions are pinned by tests/test_oracle_*.py; nothing here is
 * "parity unpinned".
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* D3Q19 velocity set, Tab. I.  Group order as in the table (rest; 6 axis     */
/* vectors; 12 diagonals).  Reading: the order inside each group is not given */
/* by the paper; opposite vectors are placed next to each other.              */
/* ------------------------------------------------------------------------- */
static const int C[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}};
static const double W[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = (dx/dt)^2 / 3, Sec. II A */

/* index of the opposite velocity: c_opp(i) = -c_i */
static const int OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static int opposite(int i) { return OPP[i]; }

void orc_d3q19(int *c, double *w, int *opp)
{
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a)
            c[3 * i + a] = C[i][a];
        w[i] = W[i];
        opp[i] = opposite(i);
    }
}

/* Equilibrium, Sec. II A:
 * f_eq_i = w_i rho [1 + (U.c_i)/cs^2 + (U.c_i)^2/(2 cs^4) - U.U/(2 cs^2)]      */
void orc_feq(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Guo source term, Sec. II A:
 * S_i = (1 - dt/(2 tau)) w_i [ (c_i - U)/cs^2 + ((U.c_i)/cs^4) c_i ] . F          */
void orc_guo_source(double tau, const double *u, const double *F, double *S)
{
    double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < 19; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += ((C[i][a] - u[a]) / CS2 + cu / (CS2 * CS2) * C[i][a]) * F[a];
        S[i] = pref * W[i] * s;
    }
}

/* One cell of the LB equation after streaming (Sec. II A, eqs. LBE, BGK,
 * hydro_var1, hydro_var2): on entry f holds the streamed populations
 * f_i(x, t); on exit the post-collision f*_i = f_i - (f_i - f_eq_i)/tau + S_i.
 * rho = sum f_i;  U = (sum c_i f_i + F dt/2) / rho (half-force correction).     */
void orc_collide_cell(double tau, const double *F, double *f, double *rho_out, double *u_out)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a)
            j[a] += C[i][a] * f[i];
    }
    double u[3];
    for (int a = 0; a < 3; ++a)
        u[a] = (j[a] + 0.5 * F[a]) / rho;
    double feq[19], S[19];
    orc_feq(rho, u, feq);
    orc_guo_source(tau, u, F, S);
    for (int i = 0; i < 19; ++i)
        f[i] = f[i] - (f[i] - feq[i]) / tau + S[i];
    *rho_out = rho;
    for (int a = 0; a < 3; ++a)
        u_out[a] = u[a];
}

/* ------------------------------------------------------------------------- */
/* Four-point kernel Psi, Sec. II A (eq. after vel_interpolation), dx = 1.   */
/* ------------------------------------------------------------------------- */
double orc_psi(double x)
{
    double r = fabs(x);
    if (r <= 1.0)
        return 0.375 - 0.25 * r + 0.25 * sqrt(r - r * r + 0.25);
    if (r <= 2.0)
        return 0.625 - 0.25 * r - 0.25 * sqrt(3.0 * r - r * r - 1.75);
    return 0.0;
}

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* wrap for a in [-n, 2n): the periodic image inside [0, n) */
static int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

static int nz_fluid(const orc_params *p) { return p->walls ? p->nz - 2 : p->nz; }

/* Fluid-layer index of full-box layer Z, or -1 when Z is solid / outside.
 * Reading (stencil at walls, silent in the paper): cells outside the fluid
 * receive no force and supply U = 0 to the interpolation; no renormalisation. */
static int fluid_layer(const orc_params *p, int Z)
{
    if (p->walls)
        return (Z >= 1 && Z <= p->nz - 2) ? Z - 1 : -1;
    return wrap(Z, p->nz);
}

/* Force spreading, eq. force_spread:  F(x) += sum_j phi_j Delta(q_j - x),
 * Delta = Psi(x) Psi(y) Psi(z) / dx^3 over the 4x4x4 support of each node.    */
void orc_spread(const orc_params *p, const double *xyz, const double *phi, int n_nodes, double *F)
{
    long cells = (long)p->nx * p->ny * nz_fluid(p);
    for (int j = 0; j < n_nodes; ++j) {
        const double *q = xyz + 3 * j;
        int b[3];
        for (int a = 0; a < 3; ++a)
            b[a] = (int)floor(q[a]);
        for (int Z = b[2] - 1; Z <= b[2] + 2; ++Z) {
            int z = fluid_layer(p, Z);
            if (z < 0)
                continue;
            double pz = orc_psi(Z - q[2]);
            for (int Y = b[1] - 1; Y <= b[1] + 2; ++Y) {
                double py = orc_psi(Y - q[1]);
                for (int X = b[0] - 1; X <= b[0] + 2; ++X) {
                    double px = orc_psi(X - q[0]);
                    long cell = wrap(X, p->nx) + (long)p->nx * (wrap(Y, p->ny) + (long)p->ny * z);
                    double d = px * py * pz;
                    for (int a = 0; a < 3; ++a)
                        F[a * cells + cell] += phi[3 * j + a] * d;
                }
            }
        }
    }
}

/* Velocity interpolation, eq. vel_interpolation:
 * qdot_j = sum_x U(x) Delta(q_j - x) dx^3, same support as the spread.        */
void orc_interp(const orc_params *p, const double *xyz, int n_nodes, const double *U, double *qdot)
{
    long cells = (long)p->nx * p->ny * nz_fluid(p);
    for (int j = 0; j < n_nodes; ++j) {
        const double *q = xyz + 3 * j;
        int b[3];
        for (int a = 0; a < 3; ++a)
            b[a] = (int)floor(q[a]);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int Z = b[2] - 1; Z <= b[2] + 2; ++Z) {
            int z = fluid_layer(p, Z);
            if (z < 0)
                continue;
            double pz = orc_psi(Z - q[2]);
            for (int Y = b[1] - 1; Y <= b[1] + 2; ++Y) {
                double py = orc_psi(Y - q[1]);
                for (int X = b[0] - 1; X <= b[0] + 2; ++X) {
                    double px = orc_psi(X - q[0]);
                    long cell = wrap(X, p->nx) + (long)p->nx * (wrap(Y, p->ny) + (long)p->ny * z);
                    double d = px * py * pz;
                    for (int a = 0; a < 3; ++a)
                        acc[a] += U[a * cells + cell] * d;
                }
            }
        }
        for (int a = 0; a < 3; ++a)
            qdot[3 * j + a] = acc[a];
    }
}

/* ------------------------------------------------------------------------- */
/* Wetting interaction, Sec. II C.                                           */
/* ------------------------------------------------------------------------- */

/* eq. A_choice: A = sigma (m-1)(n-1) / ((n-m) xi) (1 + cos theta_eq).        */
double orc_wetting_A(double sigma, double theta, double xi, int n, int m)
{
    return sigma * (double)((m - 1) * (n - 1)) / ((double)(n - m) * xi) * (1.0 + cos(theta));
}

/* eq. disjoin-p: Pi(h) = A [ (xi/h)^n - (xi/h)^m ].                          */
double orc_Pi(double h, double A, double xi, int n, int m)
{
    double r = xi / h;
    return A * (pow(r, n) - pow(r, m));
}

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void sub3(const double *a, const double *b, double *o)
{
    for (int k = 0; k < 3; ++k)
        o[k] = a[k] - b[k];
}

double orc_mesh_area(const double *xyz, const int *tri, int n_tri)
{
    double A = 0.0;
    for (int t = 0; t < n_tri; ++t) {
        double e1[3], e2[3], N[3];
        sub3(xyz + 3 * tri[3 * t + 1], xyz + 3 * tri[3 * t], e1);
        sub3(xyz + 3 * tri[3 * t + 2], xyz + 3 * tri[3 * t], e2);
        cross3(e1, e2, N);
        A += 0.5 * sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    }
    return A;
}

/* Enclosed volume of a closed outward-oriented mesh (divergence theorem):
 * V = (1/6) sum_t q_a . (q_b x q_c).                                         */
double orc_mesh_volume(const double *xyz, const int *tri, int n_tri)
{
    double V = 0.0;
    for (int t = 0; t < n_tri; ++t) {
        double bc[3];
        cross3(xyz + 3 * tri[3 * t + 1], xyz + 3 * tri[3 * t + 2], bc);
        const double *a = xyz + 3 * tri[3 * t];
        V += a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    }
    return V / 6.0;
}

/* Nodal forces phi_j = phi_sigma,j + phi_Pi,j.
 *
 * Surface tension (Sec. II B, eqs. strain_inv, energy_drop and the nodal force
 * phi_sigma,j = -dw/dV_j): for a 2x2 surface tensor M = D D^T the invariant
 * a = 1/2 log{ 1/2 [tr M]^2 - 1/2 tr(M^2) } = 1/2 log det M = log(A_t / A_t^0),
 * so w(a) = sigma e^a = sigma A_t / A_t^0.  Reading: w is an energy per unit
 * reference area (the finite-element convention of the cited thesis), so the
 * energy of triangle t is A_t^0 w = sigma A_t and the force is the exact
 * derivative  phi_sigma,j = -sigma sum_{t containing j} dA_t/dq_j,
 * dA_t/dq_a = 1/2 n_t x (q_c - q_b) for the corners (a, b, c) of t in
 * outward counter-clockwise order.  (This reproduces F_sigma = -sigma n div n.)
 *
 * Wetting (Sec. II C): phi_Pi,j = -(chi_j / 3) Pi(h_j) n_j, with
 *   n_j   = normalised average of the unit normals of the faces sharing j;
 *   chi_j = sum of the areas of the faces sharing j (each face area is
 *           shared by its three corners, hence the 1/3);
 *   h_j   = z_j - z_wall, z_wall = 1/2 (halfway bounce-back plane between the
 *           solid layer Z = 0 and the first fluid layer Z = 1).
 * Reading (silent): only the bottom wall interacts.  Reading (silent, Pi
 * diverges as h -> 0): h_eff = max(h, h_min_frac * xi); the number of nodes
 * clamped is returned.                                                       */
int orc_membrane_forces(const orc_params *p, const double *xyz, int n_nodes, const int *tri,
                        int n_tri, double *phi, double *phi_sigma, double *phi_pi)
{
    double *gs = calloc((size_t)3 * n_nodes, sizeof(double)); /* sum dA/dq */
    double *ns = calloc((size_t)3 * n_nodes, sizeof(double)); /* sum n_t   */
    double *chi = calloc((size_t)n_nodes, sizeof(double));
    for (int t = 0; t < n_tri; ++t) {
        const int *v = tri + 3 * t;
        const double *qa = xyz + 3 * v[0], *qb = xyz + 3 * v[1], *qc = xyz + 3 * v[2];
        double e1[3], e2[3], N[3];
        sub3(qb, qa, e1);
        sub3(qc, qa, e2);
        cross3(e1, e2, N);
        double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        double nh[3] = {N[0] / len, N[1] / len, N[2] / len};
        double area = 0.5 * len;
        for (int k = 0; k < 3; ++k) {
            const double *qprev = xyz + 3 * v[(k + 2) % 3];
            const double *qnext = xyz + 3 * v[(k + 1) % 3];
            double d[3], g[3];
            sub3(qprev, qnext, d);
            cross3(nh, d, g); /* dA/dq_k = 1/2 n x (q_prev - q_next) */
            for (int a = 0; a < 3; ++a) {
                gs[3 * v[k] + a] += 0.5 * g[a];
                ns[3 * v[k] + a] += nh[a];
            }
            chi[v[k]] += area;
        }
    }
    int clamped = 0;
    for (int j = 0; j < n_nodes; ++j) {
        double fs[3], fp[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a)
            fs[a] = -p->sigma * gs[3 * j + a];
        if (p->wetting) {
            double h = xyz[3 * j + 2] - 0.5;
            double hmin = p->h_min_frac * p->xi;
            if (h < hmin) {
                h = hmin;
                ++clamped;
            }
            double Pi = orc_Pi(h, p->A, p->xi, p->n, p->m);
            double nl = sqrt(ns[3 * j] * ns[3 * j] + ns[3 * j + 1] * ns[3 * j + 1] +
                             ns[3 * j + 2] * ns[3 * j + 2]);
            for (int a = 0; a < 3; ++a)
                fp[a] = -(chi[j] / 3.0) * Pi * (ns[3 * j + a] / nl);
        }
        for (int a = 0; a < 3; ++a) {
            phi[3 * j + a] = fs[a] + fp[a];
            if (phi_sigma)
                phi_sigma[3 * j + a] = fs[a];
            if (phi_pi)
                phi_pi[3 * j + a] = fp[a];
        }
    }
    free(gs);
    free(ns);
    free(chi);
    return clamped;
}

/* Elastic membrane (the strain-energy framework of Sec. II B with another
 * energy than the droplet's w = sigma e^a).  With the invariants of eq.
 * strain_inv, a = log(A / A0) and b = tr(D D^T) / 2 - 1 per triangle, the
 * Skalak energy per unit reference area is
 *   w_el = (k_s / 12) (I1^2 + 2 I1 - 2 I2) + (k_alpha / 12) I2^2,
 *   I1 = 2 b,  I2 = e^(2a) - 1,
 * and phi_j = -d/dq_j sum_t A0_t w_el(a_t, b_t) is added to phi.  The linear
 * triangle's D maps the reference edges E1, E2 (from the mesh given at set-up)
 * to the current ones e1, e2, so with the reference Gram matrix
 * H = [E_i . E_j] and S = H^-1:  tr(D D^T) = S11 e1.e1 + 2 S12 e1.e2 + S22 e2.e2,
 * A0 = sqrt(det H) / 2.  Then, with r = A / A0,
 *   phi_k = -(A0 w_a / A) dA/dq_k - A0 w_b (1/2) dtr/dq_k,
 *   A0 w_a / A = -(k_s / 3) r + (k_alpha / 3) r (r^2 - 1),   w_b = (k_s / 3)(2 b + 1),
 *   (1/2) dtr/de1 = S11 e1 + S12 e2,  (1/2) dtr/de2 = S12 e1 + S22 e2,
 * e1 = q_1 - q_0, e2 = q_2 - q_0 in the face's vertex order.                 */
void orc_membrane_elastic(const orc_params *p, const double *xyz_ref, const double *xyz, int n_nodes,
                          const int *tri, int n_tri, double *phi)
{
    (void)n_nodes;
    const double ks = p->shear_modulus, ka = p->area_modulus;
    for (int t = 0; t < n_tri; ++t) {
        const int *v = tri + 3 * t;
        double E1[3], E2[3], e1[3], e2[3], N[3];
        sub3(xyz_ref + 3 * v[1], xyz_ref + 3 * v[0], E1);
        sub3(xyz_ref + 3 * v[2], xyz_ref + 3 * v[0], E2);
        const double h11 = E1[0] * E1[0] + E1[1] * E1[1] + E1[2] * E1[2];
        const double h12 = E1[0] * E2[0] + E1[1] * E2[1] + E1[2] * E2[2];
        const double h22 = E2[0] * E2[0] + E2[1] * E2[1] + E2[2] * E2[2];
        const double det = h11 * h22 - h12 * h12;
        const double S11 = h22 / det, S12 = -h12 / det, S22 = h11 / det;
        const double A0 = 0.5 * sqrt(det);
        sub3(xyz + 3 * v[1], xyz + 3 * v[0], e1);
        sub3(xyz + 3 * v[2], xyz + 3 * v[0], e2);
        cross3(e1, e2, N);
        const double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const double A = 0.5 * len;
        const double nh[3] = {N[0] / len, N[1] / len, N[2] / len};
        const double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        const double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
        const double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
        const double b = 0.5 * (S11 * g11 + 2.0 * S12 * g12 + S22 * g22) - 1.0;
        const double r = A / A0;
        const double cA = -(ks / 3.0) * r + (ka / 3.0) * r * (r * r - 1.0);
        const double cB = A0 * (ks / 3.0) * (2.0 * b + 1.0);
        double h1[3], h2[3];     /* (1/2) dtr/de1, (1/2) dtr/de2 */
        for (int a = 0; a < 3; ++a) {
            h1[a] = S11 * e1[a] + S12 * e2[a];
            h2[a] = S12 * e1[a] + S22 * e2[a];
        }
        for (int k = 0; k < 3; ++k) {
            double d[3], gA[3];
            sub3(xyz + 3 * v[(k + 2) % 3], xyz + 3 * v[(k + 1) % 3], d);
            cross3(nh, d, gA);   /* 2 dA/dq_k */
            for (int a = 0; a < 3; ++a) {
                const double htr = k == 0 ? -(h1[a] + h2[a]) : (k == 1 ? h1[a] : h2[a]);
                phi[3 * v[k] + a] -= cA * 0.5 * gA[a] + cB * htr;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* In/out classification, Sec. II A: tau = tau_in inside the closed interface */
/* and tau_out outside, re-identified every step by ray tracing.              */
/* Reading (the paper only names "a ray tracing algorithm"): a vertical ray   */
/* through each column (X, Y); a cell is inside iff an odd number of the      */
/* mesh crossings of that ray lie strictly below the cell's Z.  A column      */
/* crosses a face iff the point lies in the face's xy projection; points on   */
/* a shared edge or vertex are assigned by a half-open rule (equivalent to a  */
/* symbolic shift of the point by (-e, -e^2)), and every edge function is     */
/* evaluated from its lower-numbered end point, so the two faces sharing an   */
/* edge see exactly opposite values and each crossing is counted once.        */
/* ------------------------------------------------------------------------- */
static double orient_edge(const double *xyz, int iu, int iv, double px, double py)
{
    int lo = iu < iv ? iu : iv, hi = iu < iv ? iv : iu;
    double ax = xyz[3 * lo], ay = xyz[3 * lo + 1];
    double bx = xyz[3 * hi], by = xyz[3 * hi + 1];
    double e = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    return iu < iv ? e : -e;
}

/* does the half-open rule keep a point lying on the directed edge u -> v? */
static int edge_keeps(const double *xyz, int iu, int iv, double s)
{
    int lo = iu < iv ? iu : iv, hi = iu < iv ? iv : iu;
    double dx = xyz[3 * hi] - xyz[3 * lo], dy = xyz[3 * hi + 1] - xyz[3 * lo + 1];
    double sg = (iu < iv ? 1.0 : -1.0) * s;
    dx *= sg;
    dy *= sg;
    return dy > 0.0 || (dy == 0.0 && dx < 0.0);
}

/* sign of the projected (doubled) area of face t, evaluated with its corners
 * in increasing index order so that it does not depend on the corner rotation */
static double face_orient(const double *xyz, const int *v)
{
    int a = v[0], b = v[1], c = v[2], par = 1, t;
    if (a > b) { t = a; a = b; b = t; par = -par; }
    if (b > c) { t = b; b = c; c = t; par = -par; }
    if (a > b) { t = a; a = b; b = t; par = -par; }
    double D = (xyz[3 * b] - xyz[3 * a]) * (xyz[3 * c + 1] - xyz[3 * a + 1]) -
               (xyz[3 * b + 1] - xyz[3 * a + 1]) * (xyz[3 * c] - xyz[3 * a]);
    return par > 0 ? D : -D;
}

typedef struct { long col; double z; } crossing;

void orc_inside(const orc_params *p, const double *xyz, const int *tri, int n_tri,
                unsigned char *inside)
{
    int nzf = nz_fluid(p);
    long ncol = (long)p->nx * p->ny;
    long cap = 64, nc = 0;
    crossing *cr = malloc(sizeof(crossing) * cap);
    for (int t = 0; t < n_tri; ++t) {
        const int *v = tri + 3 * t;
        double D = face_orient(xyz, v);
        if (D == 0.0)
            continue;
        double s = D > 0.0 ? 1.0 : -1.0;
        double xmin = xyz[3 * v[0]], xmax = xmin, ymin = xyz[3 * v[0] + 1], ymax = ymin;
        for (int k = 1; k < 3; ++k) {
            double x = xyz[3 * v[k]], y = xyz[3 * v[k] + 1];
            xmin = x < xmin ? x : xmin;
            xmax = x > xmax ? x : xmax;
            ymin = y < ymin ? y : ymin;
            ymax = y > ymax ? y : ymax;
        }
        for (int PY = (int)ceil(ymin); PY <= (int)floor(ymax); ++PY)
            for (int PX = (int)ceil(xmin); PX <= (int)floor(xmax); ++PX) {
                /* e_k: edge opposite corner k */
                double e0 = orient_edge(xyz, v[1], v[2], PX, PY);
                double e1 = orient_edge(xyz, v[2], v[0], PX, PY);
                double e2 = orient_edge(xyz, v[0], v[1], PX, PY);
                int in0 = s * e0 > 0.0 || (e0 == 0.0 && edge_keeps(xyz, v[1], v[2], s));
                int in1 = s * e1 > 0.0 || (e1 == 0.0 && edge_keeps(xyz, v[2], v[0], s));
                int in2 = s * e2 > 0.0 || (e2 == 0.0 && edge_keeps(xyz, v[0], v[1], s));
                if (!(in0 && in1 && in2))
                    continue;
                double num = (e0 * xyz[3 * v[0] + 2] + e1 * xyz[3 * v[1] + 2]) + e2 * xyz[3 * v[2] + 2];
                double den = (e0 + e1) + e2;
                if (nc == cap) {
                    cap *= 2;
                    cr = realloc(cr, sizeof(crossing) * cap);
                }
                cr[nc].col = wrap(PX, p->nx) + (long)p->nx * wrap(PY, p->ny);
                cr[nc].z = num / den;
                ++nc;
            }
    }
    for (long col = 0; col < ncol; ++col)
        for (int z = 0; z < nzf; ++z)
            inside[col + ncol * z] = 0;
    for (long k = 0; k < nc; ++k)
        for (int z = 0; z < nzf; ++z) {
            double Z = p->walls ? z + 1 : z;
            if (cr[k].z < Z)
                inside[cr[k].col + ncol * z] ^= 1;
        }
    free(cr);
}

/* ------------------------------------------------------------------------- */
/* Observables, Sec. III and App. C.                                          */
/* ------------------------------------------------------------------------- */

/* eq. angleh: tan^2(theta/2) = 3 l^3 / (R^3 - l^3); returns theta in radians. */
double orc_theta_from_height(double ell, double R)
{
    double l3 = ell * ell * ell, R3 = R * R * R;
    if (l3 >= R3)
        return M_PI;
    return 2.0 * atan(sqrt(3.0 * l3 / (R3 - l3)));
}

/* Mesh observables.  R0 is the initial radius (eq. angleh uses it); the
 * volume-equivalent radius R_V = (3V/4pi)^(1/3) is reported beside it.
 *   half-height l = (z_max - z_min)/2 (eq. ell);
 *   protocol (i) (Sec. III B): contact line = crossings of the mesh edges with
 *     the plane z = z_wall + zcut_frac*R0; r_c = mean distance of those points
 *     from their centre;  Reading: the centre of the contact plane is the mean
 *     of the crossing points; an edge crosses when one end is strictly below
 *     the plane and the other at or above it;
 *   protocol (ii): faces in the lower half (centroid below (z_min+z_max)/2)
 *     with max_ij |(q_i - q_j).z| < eps R0 are flat; chi_eps = their area,
 *     r_eps = sqrt(chi_eps / pi).                                             */
void orc_mesh_observe(const double *xyz, int n_nodes, const int *tri, int n_tri, double R0,
                      double z_wall, double zcut_frac, double eps_flat, double *out)
{
    double V = orc_mesh_volume(xyz, tri, n_tri);
    double A = orc_mesh_area(xyz, tri, n_tri);
    double c[3] = {0.0, 0.0, 0.0}, zmin = INFINITY, zmax = -INFINITY;
    for (int j = 0; j < n_nodes; ++j) {
        for (int a = 0; a < 3; ++a)
            c[a] += xyz[3 * j + a];
        zmin = fmin(zmin, xyz[3 * j + 2]);
        zmax = fmax(zmax, xyz[3 * j + 2]);
    }
    for (int a = 0; a < 3; ++a)
        c[a] /= n_nodes;
    double ell = 0.5 * (zmax - zmin);
    double RV = cbrt(3.0 * V / (4.0 * M_PI));

    /* protocol (i) */
    double zp = z_wall + zcut_frac * R0;
    double sx = 0.0, sy = 0.0;
    long ncut = 0;
    for (int pass = 0; pass < 2; ++pass) {
        double cx = ncut ? sx / ncut : 0.0, cy = ncut ? sy / ncut : 0.0, sr = 0.0;
        long cnt = 0;
        for (int t = 0; t < n_tri; ++t)
            for (int k = 0; k < 3; ++k) {
                int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
                if (a > b)
                    continue; /* every edge of a closed mesh appears once with a < b */
                double za = xyz[3 * a + 2], zb = xyz[3 * b + 2];
                if (!((za < zp && zb >= zp) || (zb < zp && za >= zp)))
                    continue;
                double s = (zp - za) / (zb - za);
                double px = xyz[3 * a] + s * (xyz[3 * b] - xyz[3 * a]);
                double py = xyz[3 * a + 1] + s * (xyz[3 * b + 1] - xyz[3 * a + 1]);
                if (pass == 0) {
                    sx += px;
                    sy += py;
                    ++ncut;
                } else {
                    sr += sqrt((px - cx) * (px - cx) + (py - cy) * (py - cy));
                    ++cnt;
                }
            }
        if (pass == 1)
            out[ORC_OBS_RC_CUT] = cnt ? sr / cnt : 0.0;
    }
    /* protocol (ii) */
    double zmid = 0.5 * (zmin + zmax), chi = 0.0;
    for (int t = 0; t < n_tri; ++t) {
        const double *qa = xyz + 3 * tri[3 * t], *qb = xyz + 3 * tri[3 * t + 1],
                     *qc = xyz + 3 * tri[3 * t + 2];
        if ((qa[2] + qb[2] + qc[2]) / 3.0 >= zmid)
            continue;
        double d = fmax(fabs(qa[2] - qb[2]), fmax(fabs(qb[2] - qc[2]), fabs(qa[2] - qc[2])));
        if (d >= eps_flat * R0)
            continue;
        double e1[3], e2[3], N[3];
        sub3(qb, qa, e1);
        sub3(qc, qa, e2);
        cross3(e1, e2, N);
        chi += 0.5 * sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    }
    out[ORC_OBS_VOLUME] = V;
    out[ORC_OBS_AREA] = A;
    out[ORC_OBS_CX] = c[0];
    out[ORC_OBS_CY] = c[1];
    out[ORC_OBS_CZ] = c[2];
    out[ORC_OBS_ZMIN] = zmin;
    out[ORC_OBS_ZMAX] = zmax;
    out[ORC_OBS_THETA_R0] = orc_theta_from_height(ell, R0) * 180.0 / M_PI;
    out[ORC_OBS_THETA_RV] = orc_theta_from_height(ell, RV) * 180.0 / M_PI;
    out[ORC_OBS_N_CUT] = (double)ncut;
    out[ORC_OBS_CHI_FLAT] = chi;
    out[ORC_OBS_RC_FLAT] = sqrt(chi / M_PI);
}

/* ------------------------------------------------------------------------- */
/* The time step.                                                             */
/* ------------------------------------------------------------------------- */
struct orc_sim {
    orc_params p;
    long cells;
    int nzf;
    double *f, *fnew;      /* 19*cells, absolute populations f*_i(x, t)      */
    double *rho, *u;       /* cells, 3*cells: moments of the last step        */
    double *F;             /* 3*cells: force density of the last step         */
    double *tau;           /* cells                                            */
    int n_nodes, n_tri;
    double *q, *phi, *qdot, *qref;
    int *tri;
    double V0, R0;
    long clamped;
};

orc_sim *orc_create(const orc_params *p)
{
    orc_sim *s = calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->nzf = nz_fluid(p);
    s->cells = (long)p->nx * p->ny * s->nzf;
    s->f = malloc(sizeof(double) * 19 * s->cells);
    s->fnew = malloc(sizeof(double) * 19 * s->cells);
    s->rho = malloc(sizeof(double) * s->cells);
    s->u = calloc((size_t)3 * s->cells, sizeof(double));
    s->F = calloc((size_t)3 * s->cells, sizeof(double));
    s->tau = malloc(sizeof(double) * s->cells);
    /* initial state: fluid at rest with density rho0, f_i = w_i rho0 (Sec. III) */
    for (int i = 0; i < 19; ++i)
        for (long c = 0; c < s->cells; ++c)
            s->f[i * s->cells + c] = W[i] * p->rho0;
    for (long c = 0; c < s->cells; ++c) {
        s->rho[c] = p->rho0;
        s->tau[c] = p->tau_out;
    }
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s)
        return;
    free(s->f);
    free(s->fnew);
    free(s->rho);
    free(s->u);
    free(s->F);
    free(s->tau);
    free(s->q);
    free(s->phi);
    free(s->qdot);
    free(s->qref);
    free(s->tri);
    free(s);
}

int orc_set_membrane(orc_sim *s, const double *xyz, int n_nodes, const int *tri, int n_tri)
{
    free(s->q);
    free(s->phi);
    free(s->qdot);
    free(s->qref);
    free(s->tri);
    s->n_nodes = n_nodes;
    s->n_tri = n_tri;
    s->q = malloc(sizeof(double) * 3 * (n_nodes ? n_nodes : 1));
    s->phi = calloc((size_t)3 * (n_nodes ? n_nodes : 1), sizeof(double));
    s->qdot = calloc((size_t)3 * (n_nodes ? n_nodes : 1), sizeof(double));
    s->tri = malloc(sizeof(int) * 3 * (n_tri ? n_tri : 1));
    s->qref = malloc(sizeof(double) * 3 * (n_nodes ? n_nodes : 1));
    memcpy(s->q, xyz, sizeof(double) * 3 * n_nodes);
    memcpy(s->qref, xyz, sizeof(double) * 3 * n_nodes);   /* the elastic reference */
    memcpy(s->tri, tri, sizeof(int) * 3 * n_tri);
    s->V0 = n_tri ? orc_mesh_volume(xyz, tri, n_tri) : 0.0;
    s->R0 = cbrt(3.0 * s->V0 / (4.0 * M_PI));
    return 0;
}

void orc_set_nodes(orc_sim *s, const double *xyz) { memcpy(s->q, xyz, sizeof(double) * 3 * s->n_nodes); }
void orc_get_nodes(const orc_sim *s, double *xyz) { memcpy(xyz, s->q, sizeof(double) * 3 * s->n_nodes); }
void orc_set_populations(orc_sim *s, const double *f) { memcpy(s->f, f, sizeof(double) * 19 * s->cells); }
void orc_get_populations(const orc_sim *s, double *f) { memcpy(f, s->f, sizeof(double) * 19 * s->cells); }
long orc_clamped_nodes(const orc_sim *s) { return s->clamped; }
long orc_cells(const orc_sim *s) { return s->cells; }

void orc_get_macros(const orc_sim *s, double *rho, double *u)
{
    memcpy(rho, s->rho, sizeof(double) * s->cells);
    memcpy(u, s->u, sizeof(double) * 3 * s->cells);
}

void orc_get_force_density(const orc_sim *s, double *F) { memcpy(F, s->F, sizeof(double) * 3 * s->cells); }
void orc_get_node_forces(const orc_sim *s, double *phi) { memcpy(phi, s->phi, sizeof(double) * 3 * s->n_nodes); }
void orc_get_tau(const orc_sim *s, double *tau) { memcpy(tau, s->tau, sizeof(double) * s->cells); }

/* One IB-LB time step.  Reading (the paper gives the ingredients, not their
 * order): the standard Guo-forced IB-LB sequence
 *   (1) nodal forces phi_j(t) from q(t)            (Sec. II B, II C)
 *   (2) F(x, t) by spreading, plus the body force  (eq. force_spread)
 *   (3) tau(x, t) from the in/out test when tau_in != tau_out (Sec. II A)
 *   (4) pull streaming with halfway bounce-back at the walls, moments with the
 *       half-force correction, BGK collision with the Guo source (eq. LBE)
 *   (5) qdot_j = interpolated U(t); q(t+1) = q(t) + qdot dt  (forward Euler)
 *   (6) optional volume correction q <- c + (q - c)(V0/V)^(1/3) about the
 *       node centroid c (not part of the paper; off unless requested).        */
static void one_step(orc_sim *s)
{
    const orc_params *p = &s->p;
    long cells = s->cells;
    int nx = p->nx, ny = p->ny, nzf = s->nzf;

    for (long k = 0; k < 3 * cells; ++k)
        s->F[k] = 0.0;
    if (s->n_nodes) {
        s->clamped = orc_membrane_forces(p, s->q, s->n_nodes, s->tri, s->n_tri, s->phi, NULL, NULL);
        if (p->shear_modulus != 0.0 || p->area_modulus != 0.0)
            orc_membrane_elastic(p, s->qref, s->q, s->n_nodes, s->tri, s->n_tri, s->phi);
        orc_spread(p, s->q, s->phi, s->n_nodes, s->F);
    }
    for (int a = 0; a < 3; ++a)
        for (long c = 0; c < cells; ++c)
            s->F[a * cells + c] += p->body_force[a];

    if (s->n_nodes && p->tau_in != p->tau_out) {
        unsigned char *in = malloc(cells);
        orc_inside(p, s->q, s->tri, s->n_tri, in);
        for (long c = 0; c < cells; ++c)
            s->tau[c] = in[c] ? p->tau_in : p->tau_out;
        free(in);
    } else {
        for (long c = 0; c < cells; ++c)
            s->tau[c] = p->tau_out;
    }

    /* every cell reads the previous populations and writes only its own
       results, so the z planes are independent: with OpenMP they are shared
       among threads, with bitwise the same results as one thread */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nzf; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long cell = x + (long)nx * (y + (long)ny * z);
                double f[19];
                for (int i = 0; i < 19; ++i) {
                    int sx = wrap1(x - C[i][0], nx), sy = wrap1(y - C[i][1], ny), sz = z - C[i][2];
                    if (p->walls && (sz < 0 || sz >= nzf)) {
                        /* halfway bounce-back at a resting wall: the population
                           that left x towards the wall comes back reversed */
                        f[i] = s->f[opposite(i) * cells + cell];
                    } else {
                        sz = wrap1(sz, nzf);
                        f[i] = s->f[i * cells + sx + (long)nx * (sy + (long)ny * sz)];
                    }
                }
                double Fc[3] = {s->F[cell], s->F[cells + cell], s->F[2 * cells + cell]};
                double rho, u[3];
                orc_collide_cell(s->tau[cell], Fc, f, &rho, u);
                for (int i = 0; i < 19; ++i)
                    s->fnew[i * cells + cell] = f[i];
                s->rho[cell] = rho;
                for (int a = 0; a < 3; ++a)
                    s->u[a * cells + cell] = u[a];
            }
    double *t = s->f;
    s->f = s->fnew;
    s->fnew = t;

    if (s->n_nodes) {
        orc_interp(p, s->q, s->n_nodes, s->u, s->qdot);
        for (long k = 0; k < 3L * s->n_nodes; ++k)
            s->q[k] += s->qdot[k];
        if (p->volume_correction) {
            double V = orc_mesh_volume(s->q, s->tri, s->n_tri);
            double c[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < s->n_nodes; ++j)
                for (int a = 0; a < 3; ++a)
                    c[a] += s->q[3 * j + a];
            for (int a = 0; a < 3; ++a)
                c[a] /= s->n_nodes;
            double k = cbrt(s->V0 / V);
            for (int j = 0; j < s->n_nodes; ++j)
                for (int a = 0; a < 3; ++a)
                    s->q[3 * j + a] = c[a] + (s->q[3 * j + a] - c[a]) * k;
        }
    }
}

/* Threads of the stream-collide loop (1 without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_step(orc_sim *s, int nsteps)
{
    for (int k = 0; k < nsteps; ++k)
        one_step(s);
}

/* mass = sum over fluid cells of sum_i f*_i (the post-collision state keeps
 * the density of the step: sum_i S_i = 0), plus the mesh observables.          */
void orc_observe(const orc_sim *s, double zcut_frac, double eps_flat, double *out)
{
    for (int k = 0; k < ORC_OBS_N; ++k)
        out[k] = 0.0;
    /* compensated (Neumaier) sum over cells of rho = sum_i f*_i, so that the
       reported mass is not limited by the rounding of a long naive sum */
    double mass = 0.0, comp = 0.0;
    for (long c = 0; c < s->cells; ++c) {
        double rho = 0.0;
        for (int i = 0; i < 19; ++i)
            rho += s->f[i * s->cells + c];
        double t = mass + rho;
        comp += fabs(mass) >= fabs(rho) ? (mass - t) + rho : (rho - t) + mass;
        mass = t;
    }
    mass += comp;
    if (s->n_nodes)
        orc_mesh_observe(s->q, s->n_nodes, s->tri, s->n_tri, s->R0, 0.5, zcut_frac, eps_flat, out);
    out[ORC_OBS_MASS] = mass;
}
