/*
 * iblb_oracle.c -- plain FP64 CPU oracle of the IBLB wetting time step.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Compile with -ffp-contract=off so that no fused
 * multiply-add changes the rounding (identical results on x86 and Arm).
 *
 * The code follows Sec. 2 of the paper in its own order and notation:
 *   Eq. 1  f_i(x + c_i, t + 1) - f_i(x, t) = Omega_i + S_i       (stream + relax)
 *   Eq. 2  Omega_i = -(f_i - f_i^eq) / tau                          (BGK)
 *   Eq. 3  f_i^eq = w_i rho [1 + u.c/cs^2 + (u.c)^2/(2cs^4) - u.u/(2cs^2)]
 *   Eq. 4  S_i = (1 - 1/(2tau)) w_i [(c_i - u)/cs^2 + (u.c_i) c_i/cs^4] . F
 *   Eq. 5-6 rho = sum f_i,  u = (sum c_i f_i + F/2) / rho
 *   Eq. 7  qdot_j = sum_x u(x) Delta(q_j - x)
 *   Eq. 8  F(x) = sum_j phi_j Delta(q_j - x)
 *   Eq. 9  interface force = surface tension + Pi(d) along the outward normal
 *   Eq. 10 Pi(d) = A[(xi/d)^n - (xi/d)^m]
 *   Eq. 11 A = sigma (m-1)(n-1) / ((n-m) xi) (1 + cos theta_eq)
 *   forward Euler q_j(t+1) = q_j(t) + qdot_j(t)                     (Sec. 2)
 *
 * Readings taken where the paper is silent (each is also listed in the design
 * notes of the repository):
 *   - D2Q9 is the 2D analogue of the paper's D3Q19; the interface is then a
 *     closed counter-clockwise ring, each segment shared by two nodes (/2
 *     instead of /3 in the nodal wetting force).
 *   - The discrete delta is Peskin's 4-point kernel.
 *   - The surface-tension force is minus sigma times the gradient of the total
 *     interface length (2D) / area (3D) with linear elements.
 *   - Solid layers: the first and last layer along the wall axis; halfway
 *     bounce-back puts the lower wall plane at 0.5; d = q_wall_axis - 0.5.
 *   - Delta stencil points on solid layers (or outside the lattice) receive no
 *     force and contribute zero velocity; no renormalisation.
 *   - Step order: forces at q(t) -> spread -> stream -> moments with F(t)
 *     -> collide -> interpolate u(t) at q(t) -> Euler.
 */
#include "iblb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CS2 (1.0 / 3.0)

/* ------------------------------------------------------------------------ */
/* Lattice stencils.  The paper does not print the weights; these are the     */
/* standard D2Q9 and D3Q19 sets (rest, axis and diagonal speeds).             */
/* ------------------------------------------------------------------------ */
int or_lattice(int Q, int* c, double* w, int* opp)
{
    static const int c9[9][2] = {
        {0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const int c19[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
        {1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};
    int i, j, k;
    if (Q == 9) {
        for (i = 0; i < 9; i++) {
            c[3 * i + 0] = c9[i][0];
            c[3 * i + 1] = c9[i][1];
            c[3 * i + 2] = 0;
            int s = abs(c9[i][0]) + abs(c9[i][1]);
            w[i] = (s == 0) ? 4.0 / 9.0 : (s == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else if (Q == 19) {
        for (i = 0; i < 19; i++) {
            for (k = 0; k < 3; k++) c[3 * i + k] = c19[i][k];
            int s = abs(c19[i][0]) + abs(c19[i][1]) + abs(c19[i][2]);
            w[i] = (s == 0) ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    } else {
        return -1;
    }
    /* opposite direction: the one with c_j = -c_i */
    for (i = 0; i < Q; i++) {
        opp[i] = -1;
        for (j = 0; j < Q; j++)
            if (c[3 * j] == -c[3 * i] && c[3 * j + 1] == -c[3 * i + 1] &&
                c[3 * j + 2] == -c[3 * i + 2])
                opp[i] = j;
    }
    return 0;
}

/* Eq. 3, with the lattice tables given */
static void equilibrium_tab(int Q, const int* c, const double* w, double rho, const double* u,
                            double* feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double uc = u[0] * c[3 * i] + u[1] * c[3 * i + 1] + u[2] * c[3 * i + 2];
        feq[i] = w[i] * rho *
                 (1.0 + uc / CS2 + (uc * uc) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 4 (dt = 1), with the lattice tables given */
static void guo_source_tab(int Q, const int* c, const double* w, double tau, const double* u,
                           const double* F, double* S)
{
    double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < Q; i++) {
        double uc = u[0] * c[3 * i] + u[1] * c[3 * i + 1] + u[2] * c[3 * i + 2];
        double s = 0.0;
        for (int a = 0; a < 3; a++) {
            double term = (c[3 * i + a] - u[a]) / CS2 + (uc / (CS2 * CS2)) * c[3 * i + a];
            s += term * F[a];
        }
        S[i] = pref * w[i] * s;
    }
}

void or_equilibrium(int Q, double rho, const double* u, double* feq)
{
    int c[19 * 3], opp[19];
    double w[19];
    or_lattice(Q, c, w, opp);
    equilibrium_tab(Q, c, w, rho, u, feq);
}

void or_guo_source(int Q, double tau, const double* u, const double* F, double* S)
{
    int c[19 * 3], opp[19];
    double w[19];
    or_lattice(Q, c, w, opp);
    guo_source_tab(Q, c, w, tau, u, F, S);
}

/* Peskin's 4-point discrete delta (one axis). */
double or_delta4(double r)
{
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* Eq. 11 */
double or_wetting_A(double sigma, double xi, double theta_eq_deg, int n, int m)
{
    double theta = theta_eq_deg * (M_PI / 180.0);
    return sigma * ((double)(m - 1) * (double)(n - 1)) / ((double)(n - m) * xi) *
           (1.0 + cos(theta));
}

static double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

/* Eq. 10 */
double or_wetting_Pi(double A, double xi, int n, int m, double d)
{
    double s = xi / d;
    return A * (ipow(s, n) - ipow(s, m));
}

/* ------------------------------------------------------------------------ */
/* Interface geometry and nodal forces (A1).                                  */
/* ------------------------------------------------------------------------ */
static void cross3(const double* a, const double* b, double* r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

int or_nodal_forces(int dim, int N, const double* q, int M, const int* tri,
                    double sigma, int wetting, double A, double xi, int n, int m,
                    double wall_plane,
                    double* phi, double* phi_sigma, double* phi_pi,
                    double* normal, double* chi)
{
    double* fs = (double*)calloc((size_t)N * 3, sizeof(double));  /* tension */
    double* nsum = (double*)calloc((size_t)N * 3, sizeof(double)); /* sum of face normals */
    double* area = (double*)calloc((size_t)N, sizeof(double));     /* 1-ring measure */
    int j, k, bad = 0;

    if (dim == 2) {
        /* closed ring: segment j joins node j and node j+1 (mod N) */
        for (j = 0; j < N; j++) {
            int jn = (j + 1) % N;
            double sx = q[2 * jn] - q[2 * j];
            double sy = q[2 * jn + 1] - q[2 * j + 1];
            double len = sqrt(sx * sx + sy * sy);
            double tx = sx / len, ty = sy / len;      /* unit tangent */
            double nux = sy / len, nuy = -sx / len;   /* outward unit normal (CCW ring) */
            /* sigma * length: d(len)/dq_j = -t, d(len)/dq_{j+1} = +t */
            fs[3 * j + 0] += sigma * tx;
            fs[3 * j + 1] += sigma * ty;
            fs[3 * jn + 0] -= sigma * tx;
            fs[3 * jn + 1] -= sigma * ty;
            nsum[3 * j + 0] += nux;
            nsum[3 * j + 1] += nuy;
            nsum[3 * jn + 0] += nux;
            nsum[3 * jn + 1] += nuy;
            area[j] += len;
            area[jn] += len;
        }
    } else {
        for (int f = 0; f < M; f++) {
            const int ia = tri[3 * f], ib = tri[3 * f + 1], ic = tri[3 * f + 2];
            const double* a = q + 3 * ia;
            const double* b = q + 3 * ib;
            const double* c = q + 3 * ic;
            double ab[3], ac[3], nf[3];
            for (k = 0; k < 3; k++) {
                ab[k] = b[k] - a[k];
                ac[k] = c[k] - a[k];
            }
            cross3(ab, ac, nf);
            double nlen = sqrt(nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2]);
            double Af = 0.5 * nlen;
            double nu[3] = {nf[0] / nlen, nf[1] / nlen, nf[2] / nlen};
            /* d(A_f)/da = 1/2 nu x (c - b), cyclic in (a, b, c) */
            const int idx[3] = {ia, ib, ic};
            const double* P[3] = {a, b, c};
            for (int v = 0; v < 3; v++) {
                const double* nxt = P[(v + 1) % 3];
                const double* prv = P[(v + 2) % 3];
                double e[3] = {prv[0] - nxt[0], prv[1] - nxt[1], prv[2] - nxt[2]};
                double g[3];
                cross3(nu, e, g);
                for (k = 0; k < 3; k++) {
                    fs[3 * idx[v] + k] -= sigma * 0.5 * g[k];
                    nsum[3 * idx[v] + k] += nu[k];
                }
                area[idx[v]] += Af;
            }
        }
    }

    const double share = (dim == 2) ? 2.0 : 3.0;
    for (j = 0; j < N; j++) {
        double nl = 0.0;
        for (k = 0; k < dim; k++) nl += nsum[3 * j + k] * nsum[3 * j + k];
        nl = sqrt(nl);
        double nh[3] = {0, 0, 0};
        for (k = 0; k < dim; k++) nh[k] = nsum[3 * j + k] / nl;
        double d = q[dim * j + dim - 1] - wall_plane;
        double pi = 0.0;
        if (wetting) {
            if (!(d > 0.0)) bad = 1;
            pi = or_wetting_Pi(A, xi, n, m, d);
        }
        for (k = 0; k < dim; k++) {
            double fpi = -area[j] * pi * nh[k] / share;
            if (phi) phi[dim * j + k] = fs[3 * j + k] + fpi;
            if (phi_sigma) phi_sigma[dim * j + k] = fs[3 * j + k];
            if (phi_pi) phi_pi[dim * j + k] = fpi;
            if (normal) normal[dim * j + k] = nh[k];
        }
        if (chi) chi[j] = area[j];
    }
    free(fs);
    free(nsum);
    free(area);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Elastic interface: Skalak strain energy on linear triangles               */
/* ------------------------------------------------------------------------ */
/* The paper forms the interface force from a finite-element strain energy
 * (Sec. 2) and names elastic interfaces as the extension to come (Sec. 5).
 * The law here is Skalak's (Skalak, Tozeren, Zarda, Chien, Biophys. J. 13,
 * 245, 1973): per unit reference area
 *   W = G_s/4 [I1^2 + 2 I1 - 2 I2 + C I2^2],
 * with the invariants I1 = tr(Cg) - 2 and I2 = det(Cg) - 1 of the in-plane
 * right Cauchy-Green tensor Cg = F^T F of each triangle (constant strain on a
 * linear triangle).  F maps the triangle's reference plane onto its current
 * position: with e1 = b - a, e2 = c - a the current edges and E1, E2 the
 * reference edges written in an orthonormal frame of the reference plane,
 * F = [e1 e2] [E1 E2]^-1. */
double or_skalak_W(double Gs, double C, double I1, double I2)
{
    return 0.25 * Gs * (I1 * I1 + 2.0 * I1 - 2.0 * I2 + C * I2 * I2);
}

void or_elastic_reference(int dim, int N, const double* q0, int M, const int* tri, double* ref)
{
    if (dim == 2) {
        for (int j = 0; j < N; j++) {
            const int jn = (j + 1) % N;
            const double sx = q0[2 * jn] - q0[2 * j], sy = q0[2 * jn + 1] - q0[2 * j + 1];
            ref[j] = sqrt(sx * sx + sy * sy);
        }
        return;
    }
    for (int f = 0; f < M; f++) {
        const double* a = q0 + 3 * tri[3 * f];
        const double* b = q0 + 3 * tri[3 * f + 1];
        const double* c = q0 + 3 * tri[3 * f + 2];
        double E1[3], E2[3], n[3], u[3], v[3];
        for (int k = 0; k < 3; k++) {
            E1[k] = b[k] - a[k];
            E2[k] = c[k] - a[k];
        }
        cross3(E1, E2, n);
        const double nlen = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const double L1 = sqrt(E1[0] * E1[0] + E1[1] * E1[1] + E1[2] * E1[2]);
        for (int k = 0; k < 3; k++) {
            u[k] = E1[k] / L1;
            n[k] /= nlen;
        }
        cross3(n, u, v);  /* in-plane unit vector perpendicular to u */
        /* reference edges in the frame (u, v): E1 -> (L1, 0), E2 -> (p, h) */
        const double p = E2[0] * u[0] + E2[1] * u[1] + E2[2] * u[2];
        const double h = E2[0] * v[0] + E2[1] * v[1] + E2[2] * v[2];
        const double det = L1 * h;
        /* inverse of [[L1, p], [0, h]] */
        ref[5 * f + 0] = h / det;
        ref[5 * f + 1] = -p / det;
        ref[5 * f + 2] = 0.0;
        ref[5 * f + 3] = L1 / det;
        ref[5 * f + 4] = 0.5 * nlen;
    }
}

double or_elastic_forces(int dim, int N, const double* q, int M, const int* tri,
                         const double* ref, double Gs, double C, double* force)
{
    double E = 0.0;
    if (force)
        for (long k = 0; k < (long)N * dim; k++) force[k] = 0.0;
    if (dim == 2) {
        /* segment j from node j to j+1, stretch lambda = l / l0, plane strain
         * (lambda2 = 1): E_j = l0 W(lambda^2 - 1, lambda^2 - 1); its tension
         * T = dE_j/dl = dW/dlambda = G_s (1 + C) lambda (lambda^2 - 1) pulls
         * node j along +t and node j+1 along -t */
        for (int j = 0; j < N; j++) {
            const int jn = (j + 1) % N;
            const double sx = q[2 * jn] - q[2 * j], sy = q[2 * jn + 1] - q[2 * j + 1];
            const double l = sqrt(sx * sx + sy * sy);
            const double lam = l / ref[j];
            const double e = lam * lam - 1.0;
            E += ref[j] * or_skalak_W(Gs, C, e, e);
            if (force) {
                const double T = Gs * (1.0 + C) * lam * e;
                force[2 * j] += T * sx / l;
                force[2 * j + 1] += T * sy / l;
                force[2 * jn] -= T * sx / l;
                force[2 * jn + 1] -= T * sy / l;
            }
        }
        return E;
    }
    for (int f = 0; f < M; f++) {
        const int ia = tri[3 * f], ib = tri[3 * f + 1], ic = tri[3 * f + 2];
        const double* Mi = ref + 5 * f;   /* Mi[2 r + c] = M_rc */
        const double A0 = ref[5 * f + 4];
        double e1[3], e2[3], F0[3], F1[3];
        for (int k = 0; k < 3; k++) {
            e1[k] = q[3 * ib + k] - q[3 * ia + k];
            e2[k] = q[3 * ic + k] - q[3 * ia + k];
        }
        /* F = [e1 e2] M: column j = e1 M_0j + e2 M_1j */
        for (int k = 0; k < 3; k++) {
            F0[k] = e1[k] * Mi[0] + e2[k] * Mi[2];
            F1[k] = e1[k] * Mi[1] + e2[k] * Mi[3];
        }
        const double C00 = F0[0] * F0[0] + F0[1] * F0[1] + F0[2] * F0[2];
        const double C01 = F0[0] * F1[0] + F0[1] * F1[1] + F0[2] * F1[2];
        const double C11 = F1[0] * F1[0] + F1[1] * F1[1] + F1[2] * F1[2];
        const double I1 = C00 + C11 - 2.0;
        const double I2 = C00 * C11 - C01 * C01 - 1.0;
        E += A0 * or_skalak_W(Gs, C, I1, I2);
        if (!force) continue;
        /* S = dW/dCg = W_1 Id + W_2 cof(Cg), W_1 = dW/dI1, W_2 = dW/dI2,
         * cof(Cg) = [[C11, -C01], [-C01, C00]] = d(det Cg)/dCg */
        const double W1 = 0.5 * Gs * (I1 + 1.0);
        const double W2 = 0.5 * Gs * (C * I2 - 1.0);
        const double S00 = W1 + W2 * C11, S01 = -W2 * C01, S11 = W1 + W2 * C00;
        /* dW/dF = 2 F S;  dW/de_k = sum_j (dW/dF)_{:,j} M_kj */
        double G0[3], G1[3], d1[3], d2[3];
        for (int k = 0; k < 3; k++) {
            G0[k] = 2.0 * (F0[k] * S00 + F1[k] * S01);
            G1[k] = 2.0 * (F0[k] * S01 + F1[k] * S11);
            d1[k] = G0[k] * Mi[0] + G1[k] * Mi[1];
            d2[k] = G0[k] * Mi[2] + G1[k] * Mi[3];
        }
        for (int k = 0; k < 3; k++) {
            force[3 * ib + k] -= A0 * d1[k];
            force[3 * ic + k] -= A0 * d2[k];
            force[3 * ia + k] += A0 * (d1[k] + d2[k]);
        }
    }
    return E;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------ */
struct or_sim {
    or_params p;
    int Q, dim;
    int c[19 * 3];
    double w[19];
    int opp[19];
    long ncell;
    int L[3];        /* extent per axis */
    int wall_axis;   /* 1 in 2D, 2 in 3D */
    double A;
    double* f;       /* post-collision populations [Q][ncell] */
    double* fnew;
    double* rho;     /* [ncell] moments of the last step */
    double* u;       /* [3][ncell] */
    double* F;       /* [3][ncell] force density */
    int N, M;
    double* q;       /* [N][dim] */
    int* tri;        /* [M][3] */
    double* phi;     /* [N][dim] */
    double* qdot;    /* [N][dim] */
    unsigned char* inside;  /* [ncell] 1 inside the interface */
    double* eref;    /* elastic reference of the interface as set (see above) */
};

static long cell_index(const or_sim* s, int x, int y, int z)
{
    return (long)x + (long)s->L[0] * ((long)y + (long)s->L[1] * (long)z);
}

/* A layer index along the wall axis is solid when walls are present and it
 * is the first or last layer, or lies outside the lattice. */
static int solid_layer(const or_sim* s, int zz)
{
    if (!s->p.walls) return 0;
    return zz <= 0 || zz >= s->L[s->wall_axis] - 1;
}

static int wrap(int i, int L)
{
    int r = i % L;
    return r < 0 ? r + L : r;
}

or_sim* or_sim_create(const or_params* p)
{
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    s->p = *p;
    s->Q = p->lattice;
    s->dim = (p->lattice == 9) ? 2 : 3;
    if (or_lattice(s->Q, s->c, s->w, s->opp) != 0) {
        free(s);
        return NULL;
    }
    s->L[0] = p->nx;
    s->L[1] = p->ny;
    s->L[2] = (s->dim == 2) ? 1 : p->nz;
    s->wall_axis = s->dim - 1;
    s->ncell = (long)s->L[0] * s->L[1] * s->L[2];
    s->A = or_wetting_A(p->sigma, p->xi, p->theta_eq_deg, p->pi_n, p->pi_m);
    s->f = (double*)malloc(sizeof(double) * s->Q * s->ncell);
    s->fnew = (double*)malloc(sizeof(double) * s->Q * s->ncell);
    s->rho = (double*)calloc(s->ncell, sizeof(double));
    s->u = (double*)calloc(3 * s->ncell, sizeof(double));
    s->F = (double*)calloc(3 * s->ncell, sizeof(double));
    s->inside = (unsigned char*)calloc(s->ncell, 1);
    /* rest state: f = w_i (rho = 1, u = 0) */
    for (int i = 0; i < s->Q; i++)
        for (long x = 0; x < s->ncell; x++) s->f[i * s->ncell + x] = s->w[i];
    for (long x = 0; x < s->ncell; x++) s->rho[x] = 1.0;
    return s;
}

void or_sim_destroy(or_sim* s)
{
    if (!s) return;
    free(s->f);
    free(s->fnew);
    free(s->rho);
    free(s->u);
    free(s->F);
    free(s->q);
    free(s->tri);
    free(s->phi);
    free(s->qdot);
    free(s->inside);
    free(s->eref);
    free(s);
}

double or_sim_A(const or_sim* s) { return s->A; }

int or_sim_set_interface(or_sim* s, int N, const double* q, int M, const int* tri)
{
    free(s->q);
    free(s->tri);
    free(s->phi);
    free(s->qdot);
    free(s->eref);
    s->eref = NULL;
    s->N = N;
    s->M = (s->dim == 3) ? M : N;
    s->q = (double*)malloc(sizeof(double) * (N > 0 ? N : 1) * s->dim);
    s->phi = (double*)calloc((N > 0 ? N : 1) * s->dim, sizeof(double));
    s->qdot = (double*)calloc((N > 0 ? N : 1) * s->dim, sizeof(double));
    s->tri = NULL;
    if (N > 0) memcpy(s->q, q, sizeof(double) * N * s->dim);
    if (s->dim == 3 && M > 0) {
        s->tri = (int*)malloc(sizeof(int) * 3 * M);
        memcpy(s->tri, tri, sizeof(int) * 3 * M);
    }
    if (N > 0 && s->p.shear_modulus != 0.0) {
        /* the interface as set is the elastic reference shape */
        s->eref = (double*)malloc(sizeof(double) * (s->dim == 3 ? 5 * (size_t)M : (size_t)N));
        or_elastic_reference(s->dim, N, s->q, s->M, s->tri, s->eref);
    }
    return 0;
}

void or_sim_set_populations(or_sim* s, const double* f)
{
    memcpy(s->f, f, sizeof(double) * s->Q * s->ncell);
}

void or_sim_set_equilibrium(or_sim* s, const double* rho, const double* u)
{
    const long nc = s->ncell;
    for (long cell = 0; cell < nc; cell++) {
        double uc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < s->dim; k++) uc[k] = u[k * nc + cell];
        double feq[19];
        equilibrium_tab(s->Q, s->c, s->w, rho ? rho[cell] : 1.0, uc, feq);
        for (int i = 0; i < s->Q; i++) s->f[i * nc + cell] = feq[i];
    }
}

void or_sim_get_populations(const or_sim* s, double* f)
{
    memcpy(f, s->f, sizeof(double) * s->Q * s->ncell);
}

void or_sim_get_fields(const or_sim* s, double* rho, double* u, double* q)
{
    if (rho) memcpy(rho, s->rho, sizeof(double) * s->ncell);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * s->ncell);
    if (q && s->N > 0) memcpy(q, s->q, sizeof(double) * s->N * s->dim);
}

static double wall_plane(const or_sim* s)
{
    (void)s;
    return 0.5; /* halfway bounce-back: lower wall plane between layers 0 and 1 */
}

int or_sim_nodal_forces(const or_sim* s, double* phi, double* normal, double* chi)
{
    const int bad = or_nodal_forces(s->dim, s->N, s->q, s->M, s->tri, s->p.sigma,
                                    s->p.wetting && s->p.walls, s->A, s->p.xi, s->p.pi_n,
                                    s->p.pi_m, wall_plane(s), phi, NULL, NULL, normal, chi);
    if (phi && s->eref) {
        /* elastic interface: add -dE/dq of the Skalak energy */
        double* fe = (double*)malloc(sizeof(double) * (size_t)s->N * s->dim);
        or_elastic_forces(s->dim, s->N, s->q, s->M, s->tri, s->eref, s->p.shear_modulus,
                          s->p.skalak_c, fe);
        for (long k = 0; k < (long)s->N * s->dim; k++) phi[k] += fe[k];
        free(fe);
    }
    return bad;
}

/* Visit the delta stencil of node position qj: calls back with the cell index
 * and the weight for every stencil point that lies on a fluid cell. */
typedef void (*stencil_fn)(long cell, double weight, void* ctx);

static void for_each_stencil_point(const or_sim* s, const double* qj, stencil_fn fn, void* ctx)
{
    int base[3] = {0, 0, 0};
    int ext[3] = {1, 1, 1};
    for (int k = 0; k < s->dim; k++) {
        base[k] = (int)floor(qj[k]) - 1;
        ext[k] = 4;
    }
    for (int c2 = 0; c2 < ext[2]; c2++)
        for (int c1 = 0; c1 < ext[1]; c1++)
            for (int c0 = 0; c0 < ext[0]; c0++) {
                int off[3] = {c0, c1, c2};
                int idx[3] = {0, 0, 0};
                double wgt = 1.0;
                int skip = 0;
                for (int k = 0; k < s->dim; k++) {
                    int ik = base[k] + off[k];
                    wgt *= or_delta4(qj[k] - (double)ik);
                    if (k == s->wall_axis && s->p.walls) {
                        if (solid_layer(s, ik)) skip = 1;
                        idx[k] = ik;
                    } else {
                        idx[k] = wrap(ik, s->L[k]);
                    }
                }
                if (skip) continue;
                fn(cell_index(s, idx[0], idx[1], idx[2]), wgt, ctx);
            }
}

typedef struct {
    double* F;
    long ncell;
    const double* phi_j;
    int dim;
} spread_ctx;

static void spread_cb(long cell, double wgt, void* vctx)
{
    spread_ctx* c = (spread_ctx*)vctx;
    for (int k = 0; k < c->dim; k++) c->F[k * c->ncell + cell] += c->phi_j[k] * wgt;
}

/* Eq. 8: F(x) += sum_j phi_j Delta(q_j - x) */
void or_sim_spread(const or_sim* s, const double* phi, double* F)
{
    spread_ctx ctx = {F, s->ncell, NULL, s->dim};
    for (int j = 0; j < s->N; j++) {
        ctx.phi_j = phi + s->dim * j;
        for_each_stencil_point(s, s->q + s->dim * j, spread_cb, &ctx);
    }
}

typedef struct {
    const double* u;
    long ncell;
    double acc[3];
    int dim;
} interp_ctx;

static void interp_cb(long cell, double wgt, void* vctx)
{
    interp_ctx* c = (interp_ctx*)vctx;
    for (int k = 0; k < c->dim; k++) c->acc[k] += c->u[k * c->ncell + cell] * wgt;
}

/* Eq. 7: qdot_j = sum_x u(x) Delta(q_j - x) (dx^3 = 1) */
void or_sim_interpolate(const or_sim* s, const double* u, double* qdot)
{
    for (int j = 0; j < s->N; j++) {
        interp_ctx ctx = {u, s->ncell, {0, 0, 0}, s->dim};
        for_each_stencil_point(s, s->q + s->dim * j, interp_cb, &ctx);
        for (int k = 0; k < s->dim; k++) qdot[s->dim * j + k] = ctx.acc[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Inside / outside classification (ray tracing, Sec. 2).  Rays run along the */
/* wall axis through the lattice columns (x in 2D; (x, y) in 3D); a cell is   */
/* inside when an odd number of interface crossings lie below it.  Ties:     */
/* a 2D segment crosses column X when min(x_a, x_b) <= X < max(x_a, x_b);    */
/* a 3D triangle, projected on the xy plane and made counter-clockwise,      */
/* covers column (X, Y) when every edge function is positive, or zero on a   */
/* top-left edge (horizontal going -x, or going -y), so that a column line   */
/* through a shared edge or vertex of a closed mesh is counted once.         */
/* Column indices wrap periodically.                                          */
/* ------------------------------------------------------------------------ */
static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double edge_fn(double ax, double ay, double bx, double by, double px, double py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

static int top_left(double ax, double ay, double bx, double by)
{
    return (ay == by && bx < ax) || (by < ay);
}

void or_sim_inside_mask(const or_sim* s, unsigned char* mask)
{
    const int dim = s->dim;
    const int ncol = (dim == 2) ? s->L[0] : s->L[0] * s->L[1];
    const int Lw = s->L[s->wall_axis];
    memset(mask, 0, (size_t)s->ncell);
    if (s->N == 0) return;
    /* crossings per column */
    int* cnt = (int*)calloc(ncol, sizeof(int));
    int cap = 64;
    double** cz = (double**)calloc(ncol, sizeof(double*));
    int* ccap = (int*)calloc(ncol, sizeof(int));
    #define OR_ADD_CROSSING(col, z)                                                   \
        do {                                                                          \
            if (cnt[col] == ccap[col]) {                                              \
                ccap[col] = ccap[col] ? 2 * ccap[col] : cap;                          \
                cz[col] = (double*)realloc(cz[col], sizeof(double) * ccap[col]);      \
            }                                                                         \
            cz[col][cnt[col]++] = (z);                                                \
        } while (0)
    if (dim == 2) {
        for (int j = 0; j < s->N; j++) {
            const int jn = (j + 1) % s->N;
            const double ax = s->q[2 * j], ay = s->q[2 * j + 1];
            const double bx = s->q[2 * jn], by = s->q[2 * jn + 1];
            const double lo = ax < bx ? ax : bx, hi = ax < bx ? bx : ax;
            for (long X = (long)ceil(lo); (double)X < hi; X++) {
                const double y = ay + ((double)X - ax) * (by - ay) / (bx - ax);
                OR_ADD_CROSSING(wrap((int)X, s->L[0]), y);
            }
        }
    } else {
        for (int f = 0; f < s->M; f++) {
            const double* P[3] = {s->q + 3 * s->tri[3 * f], s->q + 3 * s->tri[3 * f + 1],
                                  s->q + 3 * s->tri[3 * f + 2]};
            double area = edge_fn(P[0][0], P[0][1], P[1][0], P[1][1], P[2][0], P[2][1]);
            if (area == 0.0) continue; /* vertical face: no column crosses it */
            if (area < 0.0) {
                const double* t = P[1];
                P[1] = P[2];
                P[2] = t;
                area = -area;
            }
            double xmin = P[0][0], xmax = P[0][0], ymin = P[0][1], ymax = P[0][1];
            for (int k = 1; k < 3; k++) {
                if (P[k][0] < xmin) xmin = P[k][0];
                if (P[k][0] > xmax) xmax = P[k][0];
                if (P[k][1] < ymin) ymin = P[k][1];
                if (P[k][1] > ymax) ymax = P[k][1];
            }
            for (long Y = (long)ceil(ymin); (double)Y <= ymax; Y++)
                for (long X = (long)ceil(xmin); (double)X <= xmax; X++) {
                    const double px = (double)X, py = (double)Y;
                    double w[3];
                    int in = 1;
                    for (int k = 0; k < 3; k++) {
                        const double* a = P[(k + 1) % 3];
                        const double* b = P[(k + 2) % 3];
                        w[k] = edge_fn(a[0], a[1], b[0], b[1], px, py);
                        if (!(w[k] > 0.0 || (w[k] == 0.0 && top_left(a[0], a[1], b[0], b[1]))))
                            in = 0;
                    }
                    if (!in) continue;
                    /* barycentric height of the face above the column */
                    const double z = (w[0] * P[0][2] + w[1] * P[1][2] + w[2] * P[2][2]) /
                                     (w[0] + w[1] + w[2]);
                    const int col = wrap((int)X, s->L[0]) + s->L[0] * wrap((int)Y, s->L[1]);
                    OR_ADD_CROSSING(col, z);
                }
        }
    }
    #undef OR_ADD_CROSSING
    for (int col = 0; col < ncol; col++) {
        if (cnt[col] == 0) continue;
        qsort(cz[col], cnt[col], sizeof(double), cmp_double);
        for (int a = 0; a < Lw; a++) {
            int below = 0;
            for (int k = 0; k < cnt[col]; k++)
                if (cz[col][k] < (double)a) below++;
            if (below & 1) {
                long cell = (dim == 2) ? cell_index(s, col, a, 0)
                                       : cell_index(s, col % s->L[0], col / s->L[0], a);
                mask[cell] = 1;
            }
        }
        free(cz[col]);
    }
    free(cz);
    free(cnt);
    free(ccap);
}

/* Total force density of the current state: body force on fluid cells plus
 * the spread interface forces. Returns 1 if a node lies in the wall. */
static int build_force(or_sim* s)
{
    int bad = 0;
    for (int k = 0; k < 3; k++)
        for (long x = 0; x < s->ncell; x++) s->F[k * s->ncell + x] = 0.0;
    for (int z = 0; z < s->L[2]; z++)
        for (int y = 0; y < s->L[1]; y++) {
            int layer = (s->wall_axis == 1) ? y : z;
            if (solid_layer(s, layer)) continue;
            for (int x = 0; x < s->L[0]; x++) {
                long c = cell_index(s, x, y, z);
                for (int k = 0; k < 3; k++) s->F[k * s->ncell + c] = s->p.body_force[k];
            }
        }
    if (s->N > 0) {
        bad = or_sim_nodal_forces(s, s->phi, NULL, NULL);
        or_sim_spread(s, s->phi, s->F);
    }
    return bad;
}

int or_sim_force_field(or_sim* s, double* F)
{
    int bad = build_force(s);
    memcpy(F, s->F, sizeof(double) * 3 * s->ncell);
    return bad;
}

int or_sim_step(or_sim* s, int nsteps)
{
    const int Q = s->Q;
    const long nc = s->ncell;
    for (int t = 0; t < nsteps; t++) {
        /* forces at q(t), spread to F(t) */
        if (build_force(s)) return 1;
        /* viscosity ratio: inside cells relax with tau, outside with tau_out */
        const int two_tau = s->p.tau_out > 0.0 && s->p.tau_out != s->p.tau;
        if (two_tau) or_sim_inside_mask(s, s->inside);

        /* every cell is updated from the old populations alone, so the rows
         * may run in any order; a build with -fopenmp (used only to time the
         * oracle on all host cores) splits them over threads, with the same
         * arithmetic per cell */
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < s->L[2]; z++)
            for (int y = 0; y < s->L[1]; y++) {
                int layer = (s->wall_axis == 1) ? y : z;
                for (int x = 0; x < s->L[0]; x++) {
                    long cell = cell_index(s, x, y, z);
                    if (solid_layer(s, layer)) {
                        /* solid cells are not updated: they keep their populations */
                        for (int i = 0; i < Q; i++) s->fnew[i * nc + cell] = s->f[i * nc + cell];
                        s->rho[cell] = 0.0;
                        for (int k = 0; k < 3; k++) s->u[k * nc + cell] = 0.0;
                        continue;
                    }
                    /* streaming (pull) with halfway bounce-back */
                    double fi[19];
                    for (int i = 0; i < Q; i++) {
                        int src[3] = {x - s->c[3 * i], y - s->c[3 * i + 1], z - s->c[3 * i + 2]};
                        int src_layer = src[s->wall_axis];
                        if (solid_layer(s, src_layer)) {
                            /* halfway bounce-back off the wall the population
                               came from; a moving wall adds 2 w_i rho_w
                               (c_i . u_w) / c_s^2 with rho_w = 1 */
                            const double* uw = (src_layer <= 0) ? s->p.wall_u_lo : s->p.wall_u_hi;
                            const double cu = s->c[3 * i] * uw[0] + s->c[3 * i + 1] * uw[1] +
                                              s->c[3 * i + 2] * uw[2];
                            fi[i] = s->f[s->opp[i] * nc + cell] + 2.0 * s->w[i] * cu / (1.0 / 3.0);
                        } else {
                            int sx = wrap(src[0], s->L[0]);
                            int sy = wrap(src[1], s->L[1]);
                            int sz = wrap(src[2], s->L[2]);
                            fi[i] = s->f[i * nc + cell_index(s, sx, sy, sz)];
                        }
                    }
                    /* moments, Eq. 5-6 */
                    double rho = 0.0, mom[3] = {0, 0, 0};
                    for (int i = 0; i < Q; i++) {
                        rho += fi[i];
                        for (int k = 0; k < 3; k++) mom[k] += s->c[3 * i + k] * fi[i];
                    }
                    double Fc[3] = {s->F[cell], s->F[nc + cell], s->F[2 * nc + cell]};
                    double u[3];
                    for (int k = 0; k < 3; k++) u[k] = (mom[k] + 0.5 * Fc[k]) / rho;
                    /* collision, Eq. 1-4, with tau(x, t) */
                    const double tau =
                        (!two_tau || s->inside[cell]) ? s->p.tau
                                                      : (s->p.tau_out > 0.0 ? s->p.tau_out : s->p.tau);
                    double feq[19], S[19];
                    equilibrium_tab(Q, s->c, s->w, rho, u, feq);
                    guo_source_tab(Q, s->c, s->w, tau, u, Fc, S);
                    for (int i = 0; i < Q; i++)
                        s->fnew[i * nc + cell] = fi[i] - (fi[i] - feq[i]) / tau + S[i];
                    s->rho[cell] = rho;
                    for (int k = 0; k < 3; k++) s->u[k * nc + cell] = u[k];
                }
            }
        double* tmp = s->f;
        s->f = s->fnew;
        s->fnew = tmp;

        /* interpolate u(t) at q(t), then forward Euler */
        if (s->N > 0) {
            or_sim_interpolate(s, s->u, s->qdot);
            for (long j = 0; j < (long)s->N * s->dim; j++) s->q[j] += s->qdot[j];
        }
        /* non-finite check */
        for (long x = 0; x < nc; x++)
            if (!isfinite(s->rho[x])) return 2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables (A7).  The paper extracts the height as the distance between  */
/* the highest and lowest interface nodes along the wall normal.  The        */
/* contact-angle estimator (a reading, the paper gives none): algebraic      */
/* least-squares circle (2D) / sphere (3D) through the nodes with d > 3 xi,  */
/* intersected with the film plane d = min_j d_j.                            */
/* ------------------------------------------------------------------------ */
static int solve_dense(int n, double* Amat, double* b)
{
    /* Gaussian elimination with partial pivoting, Amat n x n row-major */
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(Amat[r * n + col]) > fabs(Amat[piv * n + col])) piv = r;
        if (Amat[piv * n + col] == 0.0) return 1;
        if (piv != col) {
            for (int k = 0; k < n; k++) {
                double t = Amat[col * n + k];
                Amat[col * n + k] = Amat[piv * n + k];
                Amat[piv * n + k] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < n; r++) {
            double fct = Amat[r * n + col] / Amat[col * n + col];
            for (int k = col; k < n; k++) Amat[r * n + k] -= fct * Amat[col * n + k];
            b[r] -= fct * b[col];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double acc = b[r];
        for (int k = r + 1; k < n; k++) acc -= Amat[r * n + k] * b[k];
        b[r] = acc / Amat[r * n + r];
    }
    return 0;
}

void or_sim_observables(const or_sim* s, or_obs* o)
{
    const int dim = s->dim;
    const long nc = s->ncell;
    memset(o, 0, sizeof(*o));
    /* mass: sum over fluid cells of sum_i f_i */
    double mass = 0.0;
    for (int z = 0; z < s->L[2]; z++)
        for (int y = 0; y < s->L[1]; y++) {
            int layer = (s->wall_axis == 1) ? y : z;
            if (solid_layer(s, layer)) continue;
            for (int x = 0; x < s->L[0]; x++) {
                long cell = cell_index(s, x, y, z);
                for (int i = 0; i < s->Q; i++) mass += s->f[i * nc + cell];
            }
        }
    o->mass = mass;
    const int N = s->N;
    if (N == 0) return;
    /* volume: shoelace (2D) / divergence theorem (3D) */
    double vol = 0.0;
    if (dim == 2) {
        for (int j = 0; j < N; j++) {
            int jn = (j + 1) % N;
            vol += s->q[2 * j] * s->q[2 * jn + 1] - s->q[2 * jn] * s->q[2 * j + 1];
        }
        vol *= 0.5;
    } else {
        for (int f = 0; f < s->M; f++) {
            const double* a = s->q + 3 * s->tri[3 * f];
            const double* b = s->q + 3 * s->tri[3 * f + 1];
            const double* c = s->q + 3 * s->tri[3 * f + 2];
            double bc[3];
            cross3(b, c, bc);
            vol += a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
        }
        vol /= 6.0;
    }
    o->volume = vol;
    double hmax = -1e300, hmin = 1e300;
    for (int j = 0; j < N; j++) {
        double h = s->q[dim * j + dim - 1];
        if (h > hmax) hmax = h;
        if (h < hmin) hmin = h;
    }
    o->height = hmax - hmin;
    const double wp = wall_plane(s);
    o->d_min = hmin - wp;

    /* algebraic sphere/circle fit on nodes with d > 3 xi, centred on their mean */
    double mean[3] = {0, 0, 0};
    int cnt = 0;
    for (int j = 0; j < N; j++) {
        if (s->q[dim * j + dim - 1] - wp > 3.0 * s->p.xi) {
            for (int k = 0; k < dim; k++) mean[k] += s->q[dim * j + k];
            cnt++;
        }
    }
    if (cnt < dim + 1) {
        o->theta_deg = NAN;
        o->r_cl = NAN;
        o->film = NAN;
        o->radius = NAN;
        return;
    }
    for (int k = 0; k < dim; k++) mean[k] /= cnt;
    const int np = dim + 1; /* unknowns: D_k (dim of them) and G */
    double Mt[16] = {0}, rhs[4] = {0};
    for (int j = 0; j < N; j++) {
        if (!(s->q[dim * j + dim - 1] - wp > 3.0 * s->p.xi)) continue;
        double v[4], r2 = 0.0;
        for (int k = 0; k < dim; k++) {
            v[k] = s->q[dim * j + k] - mean[k];
            r2 += v[k] * v[k];
        }
        v[dim] = 1.0;
        /* minimise sum (r2 + sum_k D_k v_k + G)^2 */
        for (int a = 0; a < np; a++) {
            for (int b = 0; b < np; b++) Mt[a * np + b] += v[a] * v[b];
            rhs[a] -= v[a] * r2;
        }
    }
    if (solve_dense(np, Mt, rhs)) {
        o->theta_deg = NAN;
        return;
    }
    double cen[3] = {0, 0, 0}, R2 = 0.0;
    for (int k = 0; k < dim; k++) {
        cen[k] = -0.5 * rhs[k];
        R2 += cen[k] * cen[k];
    }
    R2 -= rhs[dim];
    double R = sqrt(R2);
    for (int k = 0; k < dim; k++) cen[k] += mean[k];
    for (int k = 0; k < 3; k++) o->centre[k] = cen[k];
    o->radius = R;
    const double plane = wp + o->d_min; /* film plane d = eps */
    double dz = plane - cen[dim - 1];
    double cth = dz / R;
    if (cth > 1.0) cth = 1.0;
    if (cth < -1.0) cth = -1.0;
    o->theta_deg = acos(cth) * (180.0 / M_PI);
    double rcl2 = R * R - dz * dz;
    o->r_cl = rcl2 > 0.0 ? sqrt(rcl2) : 0.0;
    /* film: mean d of nodes within half the contact radius of the axis and
     * within 3 xi of the wall */
    double fsum = 0.0;
    int fc = 0;
    for (int j = 0; j < N; j++) {
        double d = s->q[dim * j + dim - 1] - wp;
        double rr = 0.0;
        for (int k = 0; k < dim - 1; k++) {
            double t = s->q[dim * j + k] - cen[k];
            rr += t * t;
        }
        if (sqrt(rr) < 0.5 * o->r_cl && d <= 3.0 * s->p.xi) {
            fsum += d;
            fc++;
        }
    }
    o->film = fc ? fsum / fc : NAN;
}

/* ------------------------------------------------------------------------ */
/* Deformation index D = (r1 - r3) / (r1 + r3) (drop in shear, Sec. 4, Eq. 15) */
/* The enclosed region is split into simplices from a reference point p0     */
/* (the node mean): triangles (p0, a, b) of the ring in 2D, tetrahedra        */
/* (p0, a, b, c) of the mesh in 3D, each with a signed measure.  Over a       */
/* simplex with vertices v_k (relative to p0) and measure |K|:                */
/*   int x dK = |K| (sum v_k) / (d + 1),                                      */
/*   int x x^T dK = |K| / ((d + 1)(d + 2)) (sum v_k v_k^T + s s^T), s = sum v_k */
/* (the vertex p0 = 0 drops out).  An ellipse with semi-axes a, b has central */
/* second moments area a^2 / 4, area b^2 / 4; an ellipsoid volume a^2 / 5 ... */
/* so the semi-axes in the shear plane (x and the wall axis) are              */
/* sqrt(4 lambda / area) (2D) and sqrt(5 lambda / volume) (3D), lambda the    */
/* eigenvalues of the central second-moment block of that plane.              */
/* ------------------------------------------------------------------------ */
void or_deformation(int dim, int N, const double* q, int M, const int* tri, double* out)
{
    double p0[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < N; j++)
        for (int k = 0; k < dim; k++) p0[k] += q[dim * j + k];
    for (int k = 0; k < dim; k++) p0[k] /= N;
    double vol = 0.0, m1[3] = {0.0, 0.0, 0.0}, m2[3][3] = {{0}};
    const int nsimp = (dim == 2) ? N : M;
    for (int t = 0; t < nsimp; t++) {
        double v[3][3] = {{0}};
        int nv;
        double meas;
        if (dim == 2) {
            const int ja = t, jb = (t + 1) % N;
            for (int k = 0; k < 2; k++) {
                v[0][k] = q[2 * ja + k] - p0[k];
                v[1][k] = q[2 * jb + k] - p0[k];
            }
            nv = 2;
            meas = 0.5 * (v[0][0] * v[1][1] - v[0][1] * v[1][0]);
        } else {
            for (int c = 0; c < 3; c++)
                for (int k = 0; k < 3; k++) v[c][k] = q[3 * tri[3 * t + c] + k] - p0[k];
            nv = 3;
            const double cx = v[1][1] * v[2][2] - v[1][2] * v[2][1];
            const double cy = v[1][2] * v[2][0] - v[1][0] * v[2][2];
            const double cz = v[1][0] * v[2][1] - v[1][1] * v[2][0];
            meas = (v[0][0] * cx + v[0][1] * cy + v[0][2] * cz) / 6.0;
        }
        double sv[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < nv; c++)
            for (int k = 0; k < 3; k++) sv[k] += v[c][k];
        vol += meas;
        for (int k = 0; k < 3; k++) m1[k] += meas * sv[k] / (dim + 1);
        const double f2 = meas / ((dim + 1) * (dim + 2));
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = sv[a] * sv[b];
                for (int c = 0; c < nv; c++) acc += v[c][a] * v[c][b];
                m2[a][b] += f2 * acc;
            }
    }
    const int w = dim - 1; /* wall axis */
    const double gx = m1[0] / vol, gw = m1[w] / vol;
    const double sxx = m2[0][0] - vol * gx * gx;
    const double sww = m2[w][w] - vol * gw * gw;
    const double sxw = m2[0][w] - vol * gx * gw;
    const double mean = 0.5 * (sxx + sww);
    const double rad = sqrt(0.25 * (sxx - sww) * (sxx - sww) + sxw * sxw);
    const double k = (dim == 2) ? 4.0 : 5.0;
    const double r1 = sqrt(k * (mean + rad) / vol);
    const double r3 = sqrt(k * (mean - rad) / vol);
    out[0] = (r1 - r3) / (r1 + r3);
    out[1] = r1;
    out[2] = r3;
    out[3] = 0.5 * atan2(2.0 * sxw, sxx - sww) * 180.0 / M_PI;
    out[4] = vol;
}
