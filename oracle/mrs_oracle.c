/*
 * mrs_oracle.c -- plain FP64 CPU oracle for the regularized-Stokeslet filament method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it (through ctypes, see oracle/__init__.py).  It shares no header, constant table or
 * helper with the CUDA path.
 *
 * Every routine is the plain definition written out, in double precision, in the order the
 * paper states it.  No blocking, no fusion, no reordering: the only parallelism is an OpenMP
 * loop over independent targets (or rods), which does not change any per-target sum.
 *
 * Paper: "Accelerating Microswimmer Simulations via a Heterogeneous Pipelined
 * Parallel-in-Time Framework".  Citations are to its sections and equations.
 *
 * Layouts (all row-major, contiguous):
 *   points      double[N][3]
 *   frames      double[N][3][3]  -- D[k][i][:] is the director D^{i+1}_k (a unit row vector)
 *   3x3 matrix  double[9]        -- M[3*r + c]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------
 * Small vector helpers (double precision).
 * ---------------------------------------------------------------------------------------- */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}

/* ==========================================================================================
 * Section II-C, Eqs. (velocity_field), (angular_velocity_field), (superposition):
 * the regularized Stokeslet / rotlet / potential-dipole pair sum.
 *
 *   mu u(x)     = f H1(r) + (f.r) r H2(r) + (n x r) H3(r)
 *   mu omega(x) = (f x r) H3(r) + n H4(r) + (n.r) r H5(r),     r = x - X_j,
 *
 * summed over every source j (the self pair r = 0 included; every H is finite there).
 * H1, H2 are the regularized Stokeslet of the blob phi_eps(r) = 15 eps^4 / (8 pi (r^2+eps^2)^{7/2})
 * (Section II-C); the paper does not print H3..H5.  They follow from omega = (1/2) curl u:
 * the rotlet H3 = (H2 - H1'/r)/2 and the dipole H4 = H3 + r H3'/2, H5 = -H3'/(2r).  The
 * CPU tests check all of them against the Stokes equations, the curl identity and the
 * singular far-field kernels, not against this code.
 * ========================================================================================== */
void orc_mrs_kernels(double r2, double eps, double* H /* [5] */)
{
    const double e2 = eps * eps;
    const double d = r2 + e2;
    const double d15 = d * sqrt(d);   /* (r^2+eps^2)^{3/2} */
    const double d25 = d15 * d;       /* (r^2+eps^2)^{5/2} */
    const double d35 = d25 * d;       /* (r^2+eps^2)^{7/2} */
    H[0] = (r2 + 2.0 * e2) / (8.0 * ORC_PI * d15);
    H[1] = 1.0 / (8.0 * ORC_PI * d15);
    H[2] = (2.0 * r2 + 5.0 * e2) / (16.0 * ORC_PI * d25);
    H[3] = (10.0 * e2 * e2 - 7.0 * e2 * r2 - 2.0 * r2 * r2) / (32.0 * ORC_PI * d35);
    H[4] = (6.0 * r2 + 21.0 * e2) / (32.0 * ORC_PI * d35);
}

/* One system: targets xt[nt][3], sources X[ns][3] carrying forces f and torques n. */
void orc_mrs_velocity(int64_t nt, const double* xt, int64_t ns, const double* X,
                      const double* f, const double* n, double eps, double mu,
                      double* u, double* w)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < nt; ++i) {
        double ui[3] = {0.0, 0.0, 0.0};
        double wi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < ns; ++j) {
            double r[3], H[5], fxr[3], nxr[3];
            r[0] = xt[3*i + 0] - X[3*j + 0];
            r[1] = xt[3*i + 1] - X[3*j + 1];
            r[2] = xt[3*i + 2] - X[3*j + 2];
            orc_mrs_kernels(dot3(r, r), eps, H);
            const double* fj = f + 3*j;
            const double* nj = n + 3*j;
            const double fr = dot3(fj, r);
            const double nr = dot3(nj, r);
            cross3(fj, r, fxr);
            cross3(nj, r, nxr);
            for (int c = 0; c < 3; ++c) {
                ui[c] += fj[c] * H[0] + fr * r[c] * H[1] + nxr[c] * H[2];
                wi[c] += fxr[c] * H[2] + nj[c] * H[3] + nr * r[c] * H[4];
            }
        }
        for (int c = 0; c < 3; ++c) {
            u[3*i + c] = ui[c] / mu;
            w[3*i + c] = wi[c] / mu;
        }
    }
}

/* Independent systems concatenated along the point axis; offsets[n_sys+1] (CSR).  Targets are
 * the sources of the same system.  eps_per_sys may be NULL (then eps applies to all). */
void orc_mrs_velocity_batch(int n_sys, const int64_t* offsets, const double* X,
                            const double* f, const double* n, double eps,
                            const double* eps_per_sys, double mu, double* u, double* w)
{
    for (int s = 0; s < n_sys; ++s) {
        const int64_t a = offsets[s], b = offsets[s + 1];
        const double e = eps_per_sys ? eps_per_sys[s] : eps;
        orc_mrs_velocity(b - a, X + 3*a, b - a, X + 3*a, f + 3*a, n + 3*a, e, mu,
                         u + 3*a, w + 3*a);
    }
}

/* ==========================================================================================
 * Section III-C-1, Eqs. (rodrigues), (halfangle): square root of a 3x3 rotation matrix.
 *
 *   cos(theta) = (tr R - 1)/2,   n = (R32-R23, R13-R31, R21-R12) / (2 sin theta),
 *   S = I cos(theta/2) + (1 - cos(theta/2)) n n^T + sin(theta/2) K(n).
 *
 * Readings where the paper leaves a choice open:
 *   - sin(theta) is taken from the length of the skew vector, theta = atan2(sin, cos), so that
 *     theta keeps full precision at both ends of [0, pi];
 *   - "theta ~ 0 => S = I" is applied only when the skew vector is exactly zero and
 *     cos(theta) > 0: any nonzero rotation keeps its half angle;
 *   - the near-pi axis estimate from the diagonal, n_i^2 = (R_ii + 1)/2, is used for every
 *     theta > pi/2 in the form n n^T = (sym(R) - cos(theta) I) / (1 - cos(theta)), which is the
 *     paper's formula at theta = pi; the largest n_i is taken positive, the other components
 *     come from the off-diagonal entries, and the overall sign is the one that agrees with the
 *     skew part.  At theta = pi exactly the result is S = R(pi/2, n), as the paper states.
 * ========================================================================================== */
void orc_rot_sqrt(const double* R, double* S)
{
    const double c = fmax(-1.0, fmin(1.0, 0.5 * (R[0] + R[4] + R[8] - 1.0)));
    const double v[3] = { R[7] - R[5], R[2] - R[6], R[3] - R[1] };
    const double sn = 0.5 * sqrt(dot3(v, v));
    double nv[3];
    if (sn == 0.0 && c > 0.0) {
        for (int q = 0; q < 9; ++q) S[q] = (q % 4 == 0) ? 1.0 : 0.0;
        return;
    }
    const double theta = atan2(sn, c);
    if (c >= 0.0) {
        for (int q = 0; q < 3; ++q) nv[q] = v[q] / (2.0 * sn);
    } else {
        double B[9];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q)
                B[3*r + q] = (0.5 * (R[3*r + q] + R[3*q + r]) - (r == q ? c : 0.0)) / (1.0 - c);
        int p = 0;
        if (B[4] > B[3*p + p]) p = 1;
        if (B[8] > B[3*p + p]) p = 2;
        const double np = sqrt(fmax(B[3*p + p], 0.0));
        for (int q = 0; q < 3; ++q) nv[q] = (q == p) ? np : B[3*p + q] / np;
        if (dot3(nv, v) < 0.0) for (int q = 0; q < 3; ++q) nv[q] = -nv[q];
        const double nn = sqrt(dot3(nv, nv));
        for (int q = 0; q < 3; ++q) nv[q] /= nn;
    }
    const double ch = cos(0.5 * theta), sh = sin(0.5 * theta);
    /* K(n) = [[0,-nz,ny],[nz,0,-nx],[-ny,nx,0]] */
    const double K[9] = { 0.0, -nv[2], nv[1], nv[2], 0.0, -nv[0], -nv[1], nv[0], 0.0 };
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q)
            S[3*r + q] = (r == q ? ch : 0.0) + (1.0 - ch) * nv[r] * nv[q] + sh * K[3*r + q];
}

/* ==========================================================================================
 * Sections II-A, II-B, IV-A: discrete Kirchhoff-rod forces and torques.
 * ========================================================================================== */
typedef struct {
    double L;        /* rod length; ds = L/(M-1) for a rod of M nodes (Section II-B) */
    double a[3];     /* bending moduli a1, a2 and torsional rigidity a3 (Eq. constitutive_N_F) */
    double b[3];     /* shear moduli b1, b2 and stretching stiffness b3 */
    double wave_A;   /* amplitude A of the preferred strain-twist wave (Section IV-A) */
    double wave_k;   /* wavenumber k = 2 pi / lambda */
    double wave_f;   /* frequency f in Omega_2 = -k^2 A sin(k s + f t) */
} orc_rod_params;

/* Omega = (0, -k^2 A sin(k s + f t), 0) (Section IV-A), evaluated at arclength s. */
static void preferred_strain(const orc_rod_params* p, double s, double t, double* Om)
{
    Om[0] = 0.0;
    Om[1] = -p->wave_k * p->wave_k * p->wave_A * sin(p->wave_k * s + p->wave_f * t);
    Om[2] = 0.0;
}

/* Segment k+1/2 of one rod (Eqs. mid_triad, F_comp_discrete, N_comp_discrete): the internal
 * force F_{k+1/2} and moment N_{k+1/2} in lab coordinates.  Xk, Xk1 are the two node
 * positions, Dk, Dk1 their frames (rows = directors), s_mid the segment's arclength.
 * Reading: Omega is evaluated at the segment midpoint; in the moment law the cyclic triple
 * (i, j, l) names the director whose arclength difference is projected, j, and the mid-frame
 * director it is projected on, l. */
static void rod_segment(const orc_rod_params* p, double ds, double s_mid, double t,
                        const double* Xk, const double* Xk1, const double* Dk, const double* Dk1,
                        double* Fseg, double* Nseg)
{
    double A[9], S[9], Dh[9], e[3], Om[3];
    /* A_k = sum_j D^j_{k+1} (D^j_k)^T */
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += Dk1[3*j + r] * Dk[3*j + q];
            A[3*r + q] = acc;
        }
    orc_rot_sqrt(A, S);
    /* D^i_{k+1/2} = A_k^{1/2} D^i_k */
    for (int i = 0; i < 3; ++i)
        for (int r = 0; r < 3; ++r)
            Dh[3*i + r] = S[3*r + 0] * Dk[3*i + 0] + S[3*r + 1] * Dk[3*i + 1] + S[3*r + 2] * Dk[3*i + 2];
    for (int q = 0; q < 3; ++q) e[q] = (Xk1[q] - Xk[q]) / ds;
    preferred_strain(p, s_mid, t, Om);
    for (int q = 0; q < 3; ++q) { Fseg[q] = 0.0; Nseg[q] = 0.0; }
    for (int jj = 0; jj < 3; ++jj) {
        /* F^j = b_j (e . D^j_{k+1/2} - delta_{3j}) */
        const double Fj = p->b[jj] * (dot3(e, Dh + 3*jj) - (jj == 2 ? 1.0 : 0.0));
        /* N^i = a_i ((D^j_{k+1} - D^j_k)/ds . D^l_{k+1/2} - Omega_i), (i, j, l) cyclic */
        const int i = jj, j = (jj + 1) % 3, l = (jj + 2) % 3;
        double dD[3];
        for (int q = 0; q < 3; ++q) dD[q] = (Dk1[3*j + q] - Dk[3*j + q]) / ds;
        const double Ni = p->a[i] * (dot3(dD, Dh + 3*l) - Om[i]);
        for (int q = 0; q < 3; ++q) {
            Fseg[q] += Fj * Dh[3*jj + q];
            Nseg[q] += Ni * Dh[3*i + q];
        }
    }
}

/* Eqs. (discrete_f), (discrete_n) for every node of every rod, returned as the point force
 * and torque the rod applies to the fluid: g_k = -f_k ds, m_k = -n_k ds (f_k, n_k are the
 * fluid-on-rod densities of Eq. momentum_balance; the fluid receives their negative).
 * Free ends: the internal force and moment beyond either end are zero and the cross term of
 * the missing segment is dropped.  rod_off[n_rods+1] are node offsets (CSR). */
void orc_rod_forces(int n_rods, const int64_t* rod_off, const double* X, const double* D,
                    const orc_rod_params* p, double t, double* g, double* m)
{
    int rr;
#pragma omp parallel for schedule(dynamic, 1)
    for (rr = 0; rr < n_rods; ++rr) {
        const int64_t a = rod_off[rr], M = rod_off[rr + 1] - rod_off[rr];
        const double ds = p->L / (double)(M - 1);
        double* Fs = (double*)malloc(sizeof(double) * 3 * (size_t)(M > 1 ? M - 1 : 1));
        double* Ns = (double*)malloc(sizeof(double) * 3 * (size_t)(M > 1 ? M - 1 : 1));
        for (int64_t k = 0; k + 1 < M; ++k)
            rod_segment(p, ds, ((double)k + 0.5) * ds, t, X + 3*(a + k), X + 3*(a + k + 1),
                        D + 9*(a + k), D + 9*(a + k + 1), Fs + 3*k, Ns + 3*k);
        for (int64_t k = 0; k < M; ++k) {
            double gk[3] = {0.0, 0.0, 0.0}, mk[3] = {0.0, 0.0, 0.0}, cr[3], dX[3];
            if (k + 1 < M) {        /* segment k+1/2 */
                for (int q = 0; q < 3; ++q) { gk[q] += Fs[3*k + q]; mk[q] += Ns[3*k + q]; }
                for (int q = 0; q < 3; ++q) dX[q] = X[3*(a + k + 1) + q] - X[3*(a + k) + q];
                cross3(dX, Fs + 3*k, cr);
                for (int q = 0; q < 3; ++q) mk[q] += 0.5 * cr[q];
            }
            if (k > 0) {            /* segment k-1/2 */
                for (int q = 0; q < 3; ++q) { gk[q] -= Fs[3*(k-1) + q]; mk[q] -= Ns[3*(k-1) + q]; }
                for (int q = 0; q < 3; ++q) dX[q] = X[3*(a + k) + q] - X[3*(a + k - 1) + q];
                cross3(dX, Fs + 3*(k-1), cr);
                for (int q = 0; q < 3; ++q) mk[q] += 0.5 * cr[q];
            }
            for (int q = 0; q < 3; ++q) { g[3*(a + k) + q] = gk[q]; m[3*(a + k) + q] = mk[q]; }
        }
        free(Fs);
        free(Ns);
    }
}

/* ==========================================================================================
 * Section III-C-3, Eqs. (newx), (newD): explicit time integration of positions and frames.
 * ========================================================================================== */

/* Eq. (newD): rotate every director of every node by theta = |omega| dt about e = omega/|omega|.
 * Reading: |omega| = 0 leaves the frame unchanged. */
void orc_rodrigues_update(int64_t N, const double* D0, const double* w, double dt, double* D1)
{
    for (int64_t k = 0; k < N; ++k) {
        const double* wk = w + 3*k;
        const double wn = sqrt(dot3(wk, wk));
        if (wn == 0.0) { memcpy(D1 + 9*k, D0 + 9*k, 9 * sizeof(double)); continue; }
        const double th = wn * dt;
        const double e[3] = { wk[0] / wn, wk[1] / wn, wk[2] / wn };
        const double ct = cos(th), st = sin(th);
        for (int i = 0; i < 3; ++i) {
            const double* Di = D0 + 9*k + 3*i;
            double exD[3];
            cross3(e, Di, exD);
            const double eD = dot3(e, Di);
            double out[3];
            for (int q = 0; q < 3; ++q) out[q] = ct * Di[q] + st * exD[q] + (1.0 - ct) * eD * e[q];
            memcpy(D1 + 9*k + 3*i, out, 3 * sizeof(double));
        }
    }
}

/* Velocities of all nodes of all rods (one hydrodynamic system, every node a source). */
static void rod_velocities(int n_rods, const int64_t* rod_off, const double* X, const double* D,
                           const orc_rod_params* p, double eps, double mu, double t,
                           double* g, double* m, double* u, double* w)
{
    const int64_t N = rod_off[n_rods];
    orc_rod_forces(n_rods, rod_off, X, D, p, t, g, m);
    orc_mrs_velocity(N, X, N, X, g, m, eps, mu, u, w);
}

/* nsteps steps of size dt from t0, in place on X[N][3] and D[N][3][3].
 * scheme 0: explicit Euler, Eqs. (newx), (newD) -- the coarse propagator G (Section III-B).
 * scheme 1: second-order Runge-Kutta -- the fine propagator F.  The paper does not name the
 *   variant; reading: the explicit midpoint rule on (X, D), with the half step taken by
 *   Eqs. (newx)/(newD) with the stage-1 velocities over dt/2, and the full step taken from the
 *   start state with the stage-2 (midpoint, time t+dt/2) velocities over dt. */
void orc_rod_step(int n_rods, const int64_t* rod_off, double* X, double* D,
                  const orc_rod_params* p, double eps, double mu, double t0, double dt,
                  int nsteps, int scheme)
{
    const int64_t N = rod_off[n_rods];
    double* g  = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* m  = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* u  = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* w  = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* Xh = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* Dh = (double*)malloc(sizeof(double) * 9 * (size_t)N);
    for (int step = 0; step < nsteps; ++step) {
        const double t = t0 + (double)step * dt;
        rod_velocities(n_rods, rod_off, X, D, p, eps, mu, t, g, m, u, w);
        if (scheme == 0) {
            for (int64_t q = 0; q < 3 * N; ++q) X[q] += u[q] * dt;
            orc_rodrigues_update(N, D, w, dt, D);
        } else {
            for (int64_t q = 0; q < 3 * N; ++q) Xh[q] = X[q] + u[q] * (0.5 * dt);
            orc_rodrigues_update(N, D, w, 0.5 * dt, Dh);
            rod_velocities(n_rods, rod_off, Xh, Dh, p, eps, mu, t + 0.5 * dt, g, m, u, w);
            for (int64_t q = 0; q < 3 * N; ++q) X[q] += u[q] * dt;
            orc_rodrigues_update(N, D, w, dt, D);
        }
    }
    free(g); free(m); free(u); free(w); free(Xh); free(Dh);
}

/* Number of OpenMP threads the oracle runs with (reported beside CPU timings). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ==========================================================================================
 * Section IV-A: Lennard-Jones repulsion between swimmers, U(r) = 4 e_lj [(sigma/r)^12 - (sigma/r)^6]
 * for r < r_c = 2^{1/6} sigma.  Readings: it acts between nodes of different rods only (nodes
 * of one rod are closer than r_c by construction); the well depth e_lj is its own parameter
 * (the paper writes it with the MRS symbol epsilon); the potential is cut at its minimum r_c,
 * so the force is purely repulsive and vanishes continuously at r_c.
 * Adds F_i = -dU/dx_i = 24 e_lj [2 (sigma/r)^12 - (sigma/r)^6] (x_i - x_j) / r^2 to F[i].
 * ========================================================================================== */
void orc_lj_forces(int64_t N, const double* X, const int* rod_id, double sigma, double e_lj,
                   double* F)
{
    const double rc2 = pow(2.0, 1.0 / 3.0) * sigma * sigma;   /* (2^{1/6} sigma)^2 */
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < N; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < N; ++j) {
            if (rod_id[i] == rod_id[j]) continue;
            double r[3];
            for (int c = 0; c < 3; ++c) r[c] = X[3*i + c] - X[3*j + c];
            const double r2 = dot3(r, r);
            if (r2 >= rc2) continue;
            const double sr2 = sigma * sigma / r2;
            const double sr6 = sr2 * sr2 * sr2;
            const double coef = 24.0 * e_lj * (2.0 * sr6 * sr6 - sr6) / r2;
            for (int c = 0; c < 3; ++c) acc[c] += coef * r[c];
        }
        for (int c = 0; c < 3; ++c) F[3*i + c] += acc[c];
    }
}
