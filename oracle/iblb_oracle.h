/*
 * iblb_oracle.h -- plain FP64 CPU oracle of the IBLB wetting time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no source with the CUDA library.
 *
 * What it computes (paper: Bellantoni et al., "On the hydrodynamic behaviour of
 * the immersed boundary - lattice Boltzmann method for wetting problems",
 * Sec. 2, "Wetting via immersed boundary - lattice Boltzmann method"):
 *   - lattice Boltzmann equation with BGK relaxation and exact streaming (Eq. 1-2),
 *   - second-order equilibrium (Eq. 3), Guo source term (Eq. 4),
 *   - moments with the half-force correction (Eq. 5-6),
 *   - IB velocity interpolation and force spreading (Eq. 7-8) with the
 *     Peskin 4-point discrete delta,
 *   - surface-tension force as the gradient of sigma * area (Eq. 9 with the
 *     finite-element strain-energy reading), wetting potential Pi(d) (Eq. 10),
 *     nodal wetting force -chi_j Pi(d_j) n_j / 3 (2D: / 2),
 *   - A from theta_eq (Eq. 11), forward-Euler node advection.
 * Readings where the paper is silent are listed with each function.
 */
#ifndef IBLB_ORACLE_H
#define IBLB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Simulation parameters.  Lattice units (dx = dt = 1). */
typedef struct {
    int lattice;          /* 9 = D2Q9 (2D), 19 = D3Q19 (3D) */
    int nx, ny, nz;       /* lattice extent; nz = 1 in 2D */
    int walls;            /* 1: the first and last layer along the wall axis
                             (y in 2D, z in 3D) are solid, halfway bounce-back;
                             0: every axis periodic */
    int wetting;          /* 1: apply Pi(d) with d measured from the lower wall */
    double tau;           /* BGK relaxation time */
    double sigma;         /* surface tension */
    double xi;            /* regularisation length of Pi */
    double theta_eq_deg;  /* equilibrium contact angle (degrees) */
    int pi_n, pi_m;       /* exponents of Pi, n > m > 1 */
    double body_force[3]; /* uniform force density on every fluid cell */
    double tau_out;       /* relaxation time outside the interface; 0 = tau
                             (viscosity ratio 1).  Inside cells use tau. */
    double wall_u_lo[3];  /* velocity of the lower / upper wall (tangential; */
    double wall_u_hi[3];  /* the wall-axis component must be 0)              */
    double shear_modulus; /* elastic interface: Skalak shear modulus G_s   */
    double skalak_c;      /* Skalak area-dilation parameter C (0 with G_s 0) */
} or_params;

/* Fixed-size observables block (every entry FP64). */
typedef struct {
    double mass;          /* sum of rho over fluid cells */
    double volume;        /* enclosed area (2D) / volume (3D) of the interface */
    double height;        /* max - min node coordinate along the wall axis */
    double theta_deg;     /* apparent contact angle of the circle/sphere fit */
    double r_cl;          /* contact-line half-width (2D) / radius (3D) */
    double film;          /* mean wall distance of the nodes under the drop */
    double d_min;         /* min wall distance over nodes */
    double centre[3];     /* fitted circle/sphere centre */
    double radius;        /* fitted radius */
} or_obs;

/* ---- pointwise pieces (for pins) ---- */
int    or_lattice(int Q, int* c /*[Q][3]*/, double* w /*[Q]*/, int* opp /*[Q]*/);
void   or_equilibrium(int Q, double rho, const double* u /*[3]*/, double* feq /*[Q]*/);
void   or_guo_source(int Q, double tau, const double* u, const double* F, double* S /*[Q]*/);
double or_delta4(double r);
double or_wetting_A(double sigma, double xi, double theta_eq_deg, int n, int m);
double or_wetting_Pi(double A, double xi, int n, int m, double d);

/* Nodal forces of an interface (A1).  dim = 2: closed CCW ring, tri ignored;
 * dim = 3: outward-oriented triangles.  Outputs are [N][dim]; any may be NULL.
 * Returns 0, or 1 if a node lies at or below the wall plane. */
int or_nodal_forces(int dim, int N, const double* q, int M, const int* tri,
                    double sigma, int wetting, double A, double xi, int n, int m,
                    double wall_plane,
                    double* phi, double* phi_sigma, double* phi_pi,
                    double* normal, double* chi);

/* ---- elastic interface (the elasticity outlook of Sec. 5; Sec. 2 forms the
 * interface force from a finite-element strain energy) ----
 * Skalak's strain energy per unit reference area of a membrane element,
 *   W = G_s/4 [I1^2 + 2 I1 - 2 I2 + C I2^2],
 *   I1 = lambda1^2 + lambda2^2 - 2,  I2 = lambda1^2 lambda2^2 - 1,
 * with lambda1, lambda2 the principal in-plane stretch ratios, on linear
 * (constant-strain) triangles whose reference shape is the interface as it
 * was set.  2D rings: the plane-strain reduction lambda2 = 1 per unit
 * reference length of each segment.  The nodal elastic force is minus the
 * gradient of the total energy. */
double or_skalak_W(double Gs, double C, double I1, double I2);
/* Reference data of an interface at positions q0: 3D, per face the inverse
 * M of the 2x2 matrix whose columns are the reference edges b - a, c - a in
 * the face's own orthonormal frame, then the reference area (5 doubles per
 * face, [M00, M01, M10, M11, A0]); 2D, per segment its reference length. */
void   or_elastic_reference(int dim, int N, const double* q0, int M, const int* tri, double* ref);
/* Total elastic energy at q; force [N][dim] (may be NULL) receives -dE/dq. */
double or_elastic_forces(int dim, int N, const double* q, int M, const int* tri,
                         const double* ref, double Gs, double C, double* force);

/* Deformation of a closed interface (the drop-in-shear test of Sec. 4, Eq. 15):
 * the second moment S of the enclosed region about its centroid, restricted
 * to the shear plane (x and the wall axis), gives the semi-axes r1 >= r3 of
 * the ellipse (2D) / ellipsoid section (3D) with the same moments, and
 * D = (r1 - r3) / (r1 + r3).  out = {D, r1, r3, inclination of the r1 axis
 * to x in degrees, enclosed area / volume}. */
void or_deformation(int dim, int N, const double* q, int M, const int* tri, double* out /*[5]*/);

/* ---- a whole simulation ---- */
typedef struct or_sim or_sim;

or_sim* or_sim_create(const or_params* p);
void    or_sim_destroy(or_sim* s);
int     or_sim_set_interface(or_sim* s, int N, const double* q, int M, const int* tri);
void    or_sim_set_populations(or_sim* s, const double* f /*[Q][cells]*/);
/* f = f_eq(rho, u) everywhere (Eq. 3); rho [cells] (NULL: 1), u [dim][cells]. */
void    or_sim_set_equilibrium(or_sim* s, const double* rho, const double* u);
void    or_sim_get_populations(const or_sim* s, double* f);
/* Advance n steps; returns 0, 1 (node in wall) or 2 (non-finite population). */
int     or_sim_step(or_sim* s, int n);
/* rho [cells], u [3][cells] of the last moment evaluation, q [N][dim]. */
void    or_sim_get_fields(const or_sim* s, double* rho, double* u, double* q);
/* Spread the nodal forces of the current interface (plus the body force) to a
 * dense force density F [3][cells]. */
int     or_sim_force_field(or_sim* s, double* F);
/* Interpolate a given velocity field u [3][cells] to the current nodes. */
void    or_sim_interpolate(const or_sim* s, const double* u, double* qdot /*[N][dim]*/);
/* Spread arbitrary nodal vectors phi [N][dim] at the current nodes. */
void    or_sim_spread(const or_sim* s, const double* phi, double* F /*[3][cells]*/);
int     or_sim_nodal_forces(const or_sim* s, double* phi, double* normal, double* chi);
/* Inside / outside classification of every cell by the current interface
 * (1 = inside), the ray-tracing step behind tau(x, t) (Sec. 2). */
void    or_sim_inside_mask(const or_sim* s, unsigned char* mask /*[cells]*/);
void    or_sim_observables(const or_sim* s, or_obs* o);
double  or_sim_A(const or_sim* s);

#ifdef __cplusplus
}
#endif
#endif
