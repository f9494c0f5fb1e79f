/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the D3Q27 central-Hermite-moment MRT lattice
 * Boltzmann method with the fully expanded equilibrium, halfway and Bouzidi bounce-back walls,
 * and velocity-inlet / pressure-outlet boundaries.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of what the
 * GPU library computes.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no source, header, table or helper with the CUDA path.
 *
 * What follows the paper (Hosseini et al., "Central moments multiple relaxation time LBM for
 * hemodynamic simulations in intracranial aneurysms"):
 *   - the lattice Boltzmann equation, collide then stream (Sec. 2.1.1, first equation);
 *   - density and momentum as the zeroth and first moments (Sec. 2.1.1);
 *   - the Hermite-expanded equilibrium, Eq. (EDF), taken to the full expansion the D3Q27
 *     stencil supports ("sixth order", Sec. 2.1.3);
 *   - the CHM-MRT operator Omega = T^-1 S T (f_eq - f) with T the central Hermite moment
 *     transform and S diagonal (Sec. 2.1.3); equilibrium central moments (rho, 0, ..., 0)
 *     (Eq. Hermite_coeff_eq); second-order rates tied to viscosity, the rest free;
 *   - the Bouzidi linear interpolated bounce-back for curved walls (Sec. 2.1.4).
 * Where the paper is silent or garbled the reading used is stated at the function (stencil
 * ordering and weights, the form of T, body forcing, the Bouzidi time levels, the inlet and
 * outlet closures, the rates of third- to sixth-order moments).
 *
 * Compiled with -O2 -ffp-contract=off; every sum runs over the directions i = 0..26 in order.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 27

/* ------------------------------------------------------------------------------------------
 * D3Q27 stencil (Sec. 2.1.3 names the stencil; the paper prints neither velocities nor
 * weights).  Reading: the standard D3Q27 set c_i in {-1,0,1}^3 numbered
 * i = (cx+1) + 3 (cy+1) + 9 (cz+1), so that the opposite direction is 26 - i, and the
 * textbook weights listed by |c|^2: 8/27, 2/27, 1/54, 1/216.  Sound speed c_s^2 = 1/3.
 * ------------------------------------------------------------------------------------------ */
static const double CS2 = 1.0 / 3.0;

static int cvel(int i, int d)
{
    int k = (d == 0) ? (i % 3) : (d == 1) ? ((i / 3) % 3) : (i / 9);
    return k - 1;
}

static int opposite(int i) { return 26 - i; }

static double weight(int i)
{
    int c2 = cvel(i, 0) * cvel(i, 0) + cvel(i, 1) * cvel(i, 1) + cvel(i, 2) * cvel(i, 2);
    switch (c2) {
    case 0: return 8.0 / 27.0;
    case 1: return 2.0 / 27.0;
    case 2: return 1.0 / 54.0;
    default: return 1.0 / 216.0;
    }
}

void oracle_stencil(int* c /* [27][3] */, double* w /* [27] */)
{
    for (int i = 0; i < NQ; ++i) {
        for (int d = 0; d < 3; ++d) c[3 * i + d] = cvel(i, d);
        w[i] = weight(i);
    }
}

/* ------------------------------------------------------------------------------------------
 * Tensor Hermite polynomials by Grad's recurrence,
 *   H_{a_1..a_n b}(x) = x_b H_{a_1..a_n}(x) - c_s^2 sum_k delta_{b a_k} H_{a_1..a_n \ a_k}(x),
 * used for the Hermite sum of Eq. (EDF).  idx holds n axis labels in {0,1,2}.
 * ------------------------------------------------------------------------------------------ */
static double hermite_tensor(int n, const int* idx, const double x[3])
{
    if (n == 0) return 1.0;
    int b = idx[n - 1];
    double v = x[b] * hermite_tensor(n - 1, idx, x);
    int sub[8];
    for (int k = 0; k < n - 1; ++k) {
        if (idx[k] != b) continue;
        int m = 0;
        for (int l = 0; l < n - 1; ++l)
            if (l != k) sub[m++] = idx[l];
        v -= CS2 * hermite_tensor(n - 2, sub, x);
    }
    return v;
}

void oracle_hermite_tensor(int n, const int* idx, const double x[3], double* out)
{
    *out = hermite_tensor(n, idx, x);
}

/* ------------------------------------------------------------------------------------------
 * Equilibrium, Eq. (EDF): f_eq_i = w_i sum_n 1/(n! c_s^{2n}) a_n^eq : H_n(c_i), with the
 * Maxwellian coefficients a_n^eq = rho u (x) ... (x) u.  "Full expansion supported by D3Q27"
 * (Sec. 2.1.3) is read as: every ordered index tuple of length n <= 6 in which no axis occurs
 * more than twice -- the tensor terms that the 27 velocities can represent, up to the xxyyzz
 * term the paper calls sixth order.
 * ------------------------------------------------------------------------------------------ */
void oracle_feq_hermite(double rho, const double u[3], double* feq)
{
    static const double fact[7] = {1, 1, 2, 6, 24, 120, 720};
    for (int i = 0; i < NQ; ++i) {
        double c[3] = {cvel(i, 0), cvel(i, 1), cvel(i, 2)};
        double sum = 0.0;
        for (int n = 0; n <= 6; ++n) {
            int ntup = 1;
            for (int k = 0; k < n; ++k) ntup *= 3;
            double cs2n = 1.0;
            for (int k = 0; k < n; ++k) cs2n *= CS2;
            for (int t = 0; t < ntup; ++t) {
                int idx[8], cnt[3] = {0, 0, 0}, tt = t;
                for (int k = 0; k < n; ++k) {
                    idx[k] = tt % 3;
                    tt /= 3;
                    cnt[idx[k]]++;
                }
                if (cnt[0] > 2 || cnt[1] > 2 || cnt[2] > 2) continue;
                double a = rho;
                for (int k = 0; k < n; ++k) a *= u[idx[k]];
                sum += a * hermite_tensor(n, idx, c) / (fact[n] * cs2n);
            }
        }
        feq[i] = weight(i) * sum;
    }
}

/* Product form of the same full expansion: f_eq_i = rho prod_d psi(c_id, u_d) with
 * psi(0,u) = 2/3 - u^2 and psi(+-1,u) = (1/3 +- u + u^2)/2, the D1Q3 distribution whose
 * first three moments are those of the Maxwellian.  The tests assert it equals
 * oracle_feq_hermite; the solver uses it because it is cheaper. */
static double psi1(int c, double u)
{
    if (c == 0) return 2.0 / 3.0 - u * u;
    return (1.0 / 3.0 + c * u + u * u) / 2.0;
}

void oracle_feq_product(double rho, const double u[3], double* feq)
{
    for (int i = 0; i < NQ; ++i)
        feq[i] = rho * psi1(cvel(i, 0), u[0]) * psi1(cvel(i, 1), u[1]) * psi1(cvel(i, 2), u[2]);
}

/* ------------------------------------------------------------------------------------------
 * Central Hermite moment transform T (Sec. 2.1.3; the paper never writes T out).  Reading:
 * a_pqr = sum_i f_i h_p(c_ix - u_x) h_q(c_iy - u_y) h_r(c_iz - u_z) with h_0 = 1, h_1 = xi,
 * h_2 = xi^2 - c_s^2, p,q,r in {0,1,2}, unnormalised so that a_000 = rho as in
 * Eq. (Hermite_coeff_eq).  Moment index m = p + 3q + 9r.  T is 27x27; T[m][i].
 * ------------------------------------------------------------------------------------------ */
static double h1d(int p, double xi)
{
    if (p == 0) return 1.0;
    if (p == 1) return xi;
    return xi * xi - CS2;
}

static int mom_p(int m, int d) { return (d == 0) ? (m % 3) : (d == 1) ? ((m / 3) % 3) : (m / 9); }
static int mom_order(int m) { return mom_p(m, 0) + mom_p(m, 1) + mom_p(m, 2); }

void oracle_chm_matrix(const double u[3], double* T)
{
    for (int m = 0; m < NQ; ++m)
        for (int i = 0; i < NQ; ++i)
            T[m * NQ + i] = h1d(mom_p(m, 0), cvel(i, 0) - u[0]) *
                            h1d(mom_p(m, 1), cvel(i, 1) - u[1]) *
                            h1d(mom_p(m, 2), cvel(i, 2) - u[2]);
}

/* T^-1.  T is the Kronecker product M(u_x) (x) M(u_y) (x) M(u_z) of the 3x3 matrices
 * M(u)[p][k] = h_p(c_k - u), so T^-1 is the Kronecker product of the three 3x3 inverses, each
 * computed by the adjugate formula.  Tinv[i][m]. */
static void inv3_of_M(double u, double inv[3][3])
{
    double M[3][3];
    for (int p = 0; p < 3; ++p)
        for (int k = 0; k < 3; ++k) M[p][k] = h1d(p, (double)(k - 1) - u);
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    /* inverse = adj(M) / det; adj(M)[k][p] = cofactor(M)[p][k] */
    for (int p = 0; p < 3; ++p)
        for (int k = 0; k < 3; ++k) {
            int r0 = (p + 1) % 3, r1 = (p + 2) % 3, c0 = (k + 1) % 3, c1 = (k + 2) % 3;
            double cof = M[r0][c0] * M[r1][c1] - M[r0][c1] * M[r1][c0];
            inv[k][p] = cof / det;
        }
}

void oracle_chm_inverse_matrix(const double u[3], double* Tinv)
{
    double ix[3][3], iy[3][3], iz[3][3];
    inv3_of_M(u[0], ix);
    inv3_of_M(u[1], iy);
    inv3_of_M(u[2], iz);
    for (int i = 0; i < NQ; ++i)
        for (int m = 0; m < NQ; ++m)
            Tinv[i * NQ + m] = ix[cvel(i, 0) + 1][mom_p(m, 0)] * iy[cvel(i, 1) + 1][mom_p(m, 1)] *
                               iz[cvel(i, 2) + 1][mom_p(m, 2)];
}

/* ------------------------------------------------------------------------------------------
 * Relaxation rates S (Sec. 2.1.3).  The six second-order moments (xx, yy, zz, xy, xz, yz) relax
 * with 1/tau (viscosity nu = c_s^2 (tau - 1/2)).  Reading for what the paper leaves free: the
 * trace (bulk) part relaxes with the same 1/tau; third- to sixth-order moments use one rate per
 * order, omega_hi[0..3] (default 1, full relaxation); the conserved zeroth- and first-order
 * rates are 1 and do not matter.
 * ------------------------------------------------------------------------------------------ */
void oracle_rates(double tau, const double omega_hi[4], double* s)
{
    for (int m = 0; m < NQ; ++m) {
        int o = mom_order(m);
        s[m] = (o <= 1) ? 1.0 : (o == 2) ? 1.0 / tau : omega_hi[o - 3];
    }
}

/* ------------------------------------------------------------------------------------------
 * CHM-MRT collision of one node (Sec. 2.1.3):
 *     f* = f + T^-1 [ S T (f_eq - f) + R ].
 * Body force (the paper's cases have none; reading for the force-driven pipe flows): a body
 * acceleration g, force density F = rho g, the velocity u = (sum_i c_i f_i)/rho + g/2 used both
 * in f_eq and in T, and the force's central Hermite moments R = (1 - s/2) F on the three
 * first-order moments and zero elsewhere (the central Hermite moments of the Maxwellian force
 * term vanish beyond first order).  With g = 0 this is exactly Omega = T^-1 S T (f_eq - f).
 * ------------------------------------------------------------------------------------------ */
void oracle_collide(const double* f, const double g[3], const double* s, double* fout)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        for (int d = 0; d < 3; ++d) j[d] += cvel(i, d) * f[i];
    }
    double u[3];
    for (int d = 0; d < 3; ++d) u[d] = j[d] / rho + 0.5 * g[d];
    double feq[NQ], T[NQ * NQ], Tinv[NQ * NQ], dm[NQ];
    oracle_feq_product(rho, u, feq);
    oracle_chm_matrix(u, T);
    oracle_chm_inverse_matrix(u, Tinv);
    for (int m = 0; m < NQ; ++m) {
        double a = 0.0;
        for (int i = 0; i < NQ; ++i) a += T[m * NQ + i] * (feq[i] - f[i]);
        dm[m] = s[m] * a;
        if (mom_order(m) == 1) {
            int d = (mom_p(m, 0) == 1) ? 0 : (mom_p(m, 1) == 1) ? 1 : 2;
            dm[m] += (1.0 - 0.5 * s[m]) * rho * g[d];
        }
    }
    for (int i = 0; i < NQ; ++i) {
        double v = 0.0;
        for (int m = 0; m < NQ; ++m) v += Tinv[i * NQ + m] * dm[m];
        fout[i] = f[i] + v;
    }
}

/* Single-relaxation-time BGK with the same (full) equilibrium, Sec. 2.1.1:
 * f* = f + (f_eq - f)/tau.  Used by the tests as the special case S = I/tau. */
void oracle_bgk(const double* f, double tau, double* fout)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        for (int d = 0; d < 3; ++d) j[d] += cvel(i, d) * f[i];
    }
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho}, feq[NQ];
    oracle_feq_product(rho, u, feq);
    for (int i = 0; i < NQ; ++i) fout[i] = f[i] + (feq[i] - f[i]) / tau;
}

/* ------------------------------------------------------------------------------------------
 * Velocity inlet / pressure outlet closure at one node (the paper only says "constant inflow at
 * the inlet" / "open boundary at the outflow" and gives an inflow curve, Sec. 2.2).  Reading: a
 * Zou-He-type closure on an axis-aligned plane with inward normal n = sign * e_axis.
 *   known:    populations with c.n <= 0;  unknown: the nine with c.n = +1.
 *   inlet:    u given; rho (1 - u.n) = sum_{c.n=0} f + 2 sum_{c.n<0} f.
 *   outlet:   rho given; u.n = 1 - (sum_{c.n=0} f + 2 sum_{c.n<0} f)/rho; tangential u = 0.
 *   unknowns: non-equilibrium bounce-back with the full equilibrium,
 *             f_i = f_opp(i) + f_eq_i(rho,u) - f_eq_opp(i)(rho,u),
 *             then for each tangential axis t, f_i += c_it D_t / 6 with
 *             D_t = rho u_t - sum_j c_jt f_j (six of the nine unknowns have c_it = +-1).
 * After the closure sum_i f_i = rho and sum_i c_i f_i = rho u hold exactly.
 * ------------------------------------------------------------------------------------------ */
void oracle_zouhe(double* f, int axis, int sign, int is_inlet, const double u_in[3], double rho_out)
{
    double s0 = 0.0, sm = 0.0;
    for (int i = 0; i < NQ; ++i) {
        int cn = cvel(i, axis) * sign;
        if (cn == 0) s0 += f[i];
        else if (cn < 0) sm += f[i];
    }
    double rho, u[3];
    if (is_inlet) {
        for (int d = 0; d < 3; ++d) u[d] = u_in[d];
        rho = (s0 + 2.0 * sm) / (1.0 - u[axis] * sign);
    } else {
        rho = rho_out;
        for (int d = 0; d < 3; ++d) u[d] = 0.0;
        u[axis] = sign * (1.0 - (s0 + 2.0 * sm) / rho);
    }
    double feq[NQ];
    oracle_feq_product(rho, u, feq);
    for (int i = 0; i < NQ; ++i)
        if (cvel(i, axis) * sign == 1) f[i] = f[opposite(i)] + feq[i] - feq[opposite(i)];
    double D[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < 3; ++t) {
        if (t == axis) continue;
        double mom = 0.0;
        for (int j = 0; j < NQ; ++j) mom += cvel(j, t) * f[j];
        D[t] = rho * u[t] - mom;
    }
    for (int t = 0; t < 3; ++t) {
        if (t == axis) continue;
        for (int i = 0; i < NQ; ++i)
            if (cvel(i, axis) * sign == 1) f[i] += cvel(i, t) * D[t] / 6.0;
    }
}

/* ------------------------------------------------------------------------------------------
 * Inflow waveform (the paper gives an inflow curve over one cycle, Sec. 2.2; the synthetic cases
 * use a Fourier series):  s(t) = a_0 + sum_k a_k cos(2 pi k t/P) + b_k sin(2 pi k t/P),
 * U(t) = u_peak s(t) / max_{t in 0..P-1} s(t), the maximum taken over integer steps.  With no
 * harmonics U = u_peak a_0 / a_0 = u_peak.
 * ------------------------------------------------------------------------------------------ */
static double wave_s(const double* a, const double* b, int nh, double P, double t)
{
    const double two_pi = 6.283185307179586476925286766559;
    double s = a[0];
    for (int k = 1; k <= nh; ++k) {
        double ph = two_pi * k * t / P;
        s += a[k] * cos(ph) + b[k - 1] * sin(ph);
    }
    return s;
}

double oracle_waveform(const double* a, const double* b, int nh, double P, double u_peak, double t)
{
    double smax = -INFINITY;
    for (long k = 0; k < (long)P; ++k) {
        double v = wave_s(a, b, nh, P, (double)k);
        if (v > smax) smax = v;
    }
    return u_peak * wave_s(a, b, nh, P, t) / smax;
}

/* ------------------------------------------------------------------------------------------
 * The classical operators the paper compares against (Sec. 2.1.2): the single-relaxation-time
 * (SRT, BGK) operator with the second-order equilibrium, and the two-relaxation-time (TRT)
 * operator it cites as the fix for the viscosity-dependent wall position of bounce-back.  The
 * paper prints neither; the readings are the textbook forms.
 *   Second-order equilibrium: the Hermite expansion of Eq. (EDF) truncated after the
 *   second-order term, f_eq2_i = w_i rho [1 + c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)].
 *   Body force (as for the CHM-MRT operator: u = sum c f / rho + g/2, F = rho g): the
 *   second-order force term of Guo, Zheng and Shi (2002),
 *     F_i = w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . F,
 *   whose odd part is w_i c_i.F / c_s^2 and whose even part is the rest.
 *   SRT:  f* = f + (f_eq2 - f)/tau + (1 - 1/(2 tau)) F_i.
 *   TRT (Ginzburg): even / odd parts p_i = (f_i + f_opp(i))/2, m_i = (f_i - f_opp(i))/2 relax with
 *     w+ = 1/tau and w- = 1/(Lambda/(tau - 1/2) + 1/2), Lambda the "magic" parameter;
 *     f* = f - w+ (p - p_eq) - w- (m - m_eq) + (1 - w+/2) F_even + (1 - w-/2) F_odd.
 *   Lambda = (tau - 1/2)^2 gives w- = w+ and the SRT operator.
 * ------------------------------------------------------------------------------------------ */
void oracle_feq2(double rho, const double u[3], double* feq)
{
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NQ; ++i) {
        double cu = 0.0;
        for (int d = 0; d < 3; ++d) cu += cvel(i, d) * u[d];
        feq[i] = weight(i) * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Guo force term split into its even and odd parts (both without the (1 - w/2) factor). */
static void guo_force(const double u[3], const double F[3], double* Feven, double* Fodd)
{
    for (int i = 0; i < NQ; ++i) {
        double cu = 0.0, cF = 0.0, uF = 0.0;
        for (int d = 0; d < 3; ++d) {
            cu += cvel(i, d) * u[d];
            cF += cvel(i, d) * F[d];
            uF += u[d] * F[d];
        }
        Fodd[i] = weight(i) * cF / CS2;
        Feven[i] = weight(i) * (-uF / CS2 + cu * cF / (CS2 * CS2));
    }
}

static void moments_rho_u(const double* f, const double g[3], double* rho, double u[3])
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        r += f[i];
        for (int d = 0; d < 3; ++d) j[d] += cvel(i, d) * f[i];
    }
    *rho = r;
    for (int d = 0; d < 3; ++d) u[d] = j[d] / r + 0.5 * g[d];
}

void oracle_collide_srt2(const double* f, const double g[3], double tau, double* fout)
{
    double rho, u[3], feq[NQ], Fe[NQ], Fo[NQ];
    moments_rho_u(f, g, &rho, u);
    const double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
    oracle_feq2(rho, u, feq);
    guo_force(u, F, Fe, Fo);
    const double w = 1.0 / tau;
    for (int i = 0; i < NQ; ++i) fout[i] = f[i] + w * (feq[i] - f[i]) + (1.0 - 0.5 * w) * (Fe[i] + Fo[i]);
}

double oracle_trt_minus_rate(double tau, double magic) { return 1.0 / (magic / (tau - 0.5) + 0.5); }

void oracle_collide_trt2(const double* f, const double g[3], double tau, double magic, double* fout)
{
    double rho, u[3], feq[NQ], Fe[NQ], Fo[NQ];
    moments_rho_u(f, g, &rho, u);
    const double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
    oracle_feq2(rho, u, feq);
    guo_force(u, F, Fe, Fo);
    const double wp = 1.0 / tau, wm = oracle_trt_minus_rate(tau, magic);
    for (int i = 0; i < NQ; ++i) {
        const int o = opposite(i);
        const double p = 0.5 * (f[i] + f[o]), m = 0.5 * (f[i] - f[o]);
        const double peq = 0.5 * (feq[i] + feq[o]), meq = 0.5 * (feq[i] - feq[o]);
        fout[i] = f[i] - wp * (p - peq) - wm * (m - meq) + (1.0 - 0.5 * wp) * Fe[i] + (1.0 - 0.5 * wm) * Fo[i];
    }
}

/* ------------------------------------------------------------------------------------------
 * A whole case on a voxel box (Sec. 2.1.1 LBE; Sec. 2.1.4 walls; Sec. 2.2 boundaries).
 *   mask (x fastest): 0 solid, 1 fluid, 2 inlet, 3 outlet.  Cells outside a non-periodic face
 *   count as solid.  Inlet/outlet cells lie on exactly one non-periodic box face, whose inward
 *   normal is theirs.
 *   links: (fluid cell, beta, q): x_f + c_beta is not fluid and the wall cuts that link at
 *   q |c_beta| from x_f, q in (0, 1].  Wall links without a q use halfway bounce-back.
 * State: f(x, n), the populations after streaming and boundary closures at time level n.
 * One step n -> n+1: collide every fluid node with g(n); stream by the LBE (written in pull
 * form: f_i(x, n+1) = f*_i(x - c_i, n)) with the wall rule where x - c_i is not fluid; then the
 * inlet/outlet closures at time n+1.  The initial state is f = w (rho = 1, u = 0) followed by the
 * closures at n = 0.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz, periodic[3];
    int64_t nfluid;
    int32_t* map;     /* box index -> fluid index, -1 for solid */
    int64_t* cell;    /* fluid index -> box index (increasing) */
    uint8_t* kind;    /* 1 fluid, 2 inlet, 3 outlet */
    int8_t* naxis;    /* inward normal axis of inlet/outlet cells */
    int8_t* nsign;
    double* phi;      /* inlet profile factor 2 (1 - r^2/R^2), >= 0 */
    double* qlink;    /* [nfluid][27], q of the wall link whose unknown is direction i; 0 = none */
    double *f, *fpost;
    double s[NQ];
    double* tau_cell; /* [nfluid] relaxation time of each cell (NULL: tau everywhere) */
    double omega_hi[4];
    double g0[3], gamp[3], gomega, rho_out;
    double wa[16], wb[16], wP, wpeak;
    int wnh, has_wave;
    int collision;    /* 0 CHM-MRT, 1 SRT with f_eq2, 2 TRT with f_eq2 */
    double tau, magic;
    int64_t n;
} oracle_case;

static void set_err(char* err, int len, const char* msg)
{
    if (err && len > 0) {
        strncpy(err, msg, (size_t)len - 1);
        err[len - 1] = 0;
    }
}

/* source node of direction i pulled into (x,y,z) shifted by sgn*c_i; returns fluid index or -1 */
static int64_t shifted(const oracle_case* C, int x, int y, int z, int i, int sgn)
{
    int p[3] = {x + sgn * cvel(i, 0), y + sgn * cvel(i, 1), z + sgn * cvel(i, 2)};
    int n[3] = {C->nx, C->ny, C->nz};
    for (int d = 0; d < 3; ++d) {
        if (p[d] < 0 || p[d] >= n[d]) {
            if (!C->periodic[d]) return -1;
            p[d] = (p[d] + n[d]) % n[d];
        }
    }
    int64_t b = (int64_t)p[0] + (int64_t)C->nx * ((int64_t)p[1] + (int64_t)C->ny * p[2]);
    return C->map[b];
}

static void gforce(const oracle_case* C, int64_t n, double g[3])
{
    for (int d = 0; d < 3; ++d) g[d] = C->g0[d] + C->gamp[d] * cos(C->gomega * (double)n);
}

static double inlet_U(const oracle_case* C, int64_t n)
{
    if (!C->has_wave) return 0.0;
    double t = fmod((double)n, C->wP);
    return oracle_waveform(C->wa, C->wb, C->wnh, C->wP, C->wpeak, t);
}

static void apply_open_boundaries(oracle_case* C, int64_t n)
{
    double U = inlet_U(C, n);
    for (int64_t k = 0; k < C->nfluid; ++k) {
        if (C->kind[k] < 2) continue;
        double u[3] = {0.0, 0.0, 0.0};
        int ax = C->naxis[k], sg = C->nsign[k];
        u[ax] = sg * U * C->phi[k];
        oracle_zouhe(C->f + k * NQ, ax, sg, C->kind[k] == 2, u, C->rho_out);
    }
}

static void stream(oracle_case* C);

void oracle_destroy(oracle_case* C)
{
    if (!C) return;
    free(C->map);
    free(C->cell);
    free(C->kind);
    free(C->naxis);
    free(C->nsign);
    free(C->phi);
    free(C->qlink);
    free(C->f);
    free(C->fpost);
    free(C->tau_cell);
    free(C);
}

oracle_case* oracle_create(int nx, int ny, int nz, const uint8_t* mask, const int* periodic,
                           const int64_t* link_cell, const uint8_t* link_dir, const double* link_q,
                           int64_t n_links, const double* inlet_center, double inlet_radius,
                           double tau, const double* omega_hi, const double* g0, const double* gamp,
                           double gomega, double rho_out, const double* tau_box, char* err, int errlen)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || tau <= 0.5) {
        set_err(err, errlen, "bad box size or tau <= 1/2");
        return NULL;
    }
    oracle_case* C = (oracle_case*)calloc(1, sizeof(oracle_case));
    C->nx = nx;
    C->ny = ny;
    C->nz = nz;
    for (int d = 0; d < 3; ++d) C->periodic[d] = periodic[d] ? 1 : 0;
    int64_t nbox = (int64_t)nx * ny * nz;
    C->map = (int32_t*)malloc(sizeof(int32_t) * nbox);
    int64_t nf = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        if (mask[b] > 3) {
            set_err(err, errlen, "mask value > 3");
            oracle_destroy(C);
            return NULL;
        }
        C->map[b] = mask[b] ? (int32_t)nf++ : -1;
    }
    C->nfluid = nf;
    C->cell = (int64_t*)malloc(sizeof(int64_t) * (nf ? nf : 1));
    C->kind = (uint8_t*)malloc(nf ? nf : 1);
    C->naxis = (int8_t*)calloc(nf ? nf : 1, 1);
    C->nsign = (int8_t*)calloc(nf ? nf : 1, 1);
    C->phi = (double*)calloc(nf ? nf : 1, sizeof(double));
    C->qlink = (double*)calloc((size_t)(nf ? nf : 1) * NQ, sizeof(double));
    C->f = (double*)malloc(sizeof(double) * (size_t)(nf ? nf : 1) * NQ);
    C->fpost = (double*)malloc(sizeof(double) * (size_t)(nf ? nf : 1) * NQ);
    int n3[3] = {nx, ny, nz};
    for (int64_t b = 0; b < nbox; ++b) {
        if (C->map[b] < 0) continue;
        int64_t k = C->map[b];
        C->cell[k] = b;
        C->kind[k] = mask[b];
        if (mask[b] >= 2) {
            int p[3] = {(int)(b % nx), (int)((b / nx) % ny), (int)(b / ((int64_t)nx * ny))};
            int faces = 0, ax = -1, sg = 0;
            for (int d = 0; d < 3; ++d) {
                if (C->periodic[d]) continue;
                if (p[d] == 0) { faces++; ax = d; sg = +1; }
                if (p[d] == n3[d] - 1) { faces++; ax = d; sg = -1; }
            }
            if (faces != 1) {
                set_err(err, errlen, "inlet/outlet cell not on exactly one non-periodic face");
                oracle_destroy(C);
                return NULL;
            }
            C->naxis[k] = (int8_t)ax;
            C->nsign[k] = (int8_t)sg;
            if (mask[b] == 2) {
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    if (d == ax) continue;
                    double dx = p[d] + 0.5 - inlet_center[d];
                    r2 += dx * dx;
                }
                double v = 2.0 * (1.0 - r2 / (inlet_radius * inlet_radius));
                C->phi[k] = v > 0.0 ? v : 0.0;
            }
        }
    }
    for (int64_t l = 0; l < n_links; ++l) {
        int64_t b = link_cell[l];
        int beta = link_dir[l];
        double q = link_q[l];
        if (b < 0 || b >= nbox || beta >= NQ || beta == 13 || !(q > 0.0 && q <= 1.0)) {
            set_err(err, errlen, "link out of range");
            oracle_destroy(C);
            return NULL;
        }
        int64_t k = C->map[b];
        if (k < 0 || C->kind[k] != 1) {
            set_err(err, errlen, "link cell is not a plain fluid cell");
            oracle_destroy(C);
            return NULL;
        }
        int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / ((int64_t)nx * ny));
        if (shifted(C, x, y, z, beta, +1) >= 0) {
            set_err(err, errlen, "link does not point into a wall");
            oracle_destroy(C);
            return NULL;
        }
        int alpha = opposite(beta);
        if (C->qlink[k * NQ + alpha] != 0.0) {
            set_err(err, errlen, "duplicate link");
            oracle_destroy(C);
            return NULL;
        }
        C->qlink[k * NQ + alpha] = q;
    }
    oracle_rates(tau, omega_hi, C->s);
    for (int k = 0; k < 4; ++k) C->omega_hi[k] = omega_hi[k];
    C->tau = tau;
    C->collision = 0;
    C->magic = 3.0 / 16.0;
    /* an optional relaxation time per cell (a viscosity field, e.g. an absorbing layer before an
     * outlet); the second-order rate of the cell is then 1/tau_cell */
    if (tau_box) {
        C->tau_cell = (double*)malloc(sizeof(double) * (size_t)(nf ? nf : 1));
        for (int64_t k = 0; k < nf; ++k) {
            double t = tau_box[C->cell[k]];
            if (!(t > 0.5)) {
                set_err(err, errlen, "tau_cell must be > 1/2 at fluid cells");
                oracle_destroy(C);
                return NULL;
            }
            C->tau_cell[k] = t;
        }
    }
    for (int d = 0; d < 3; ++d) {
        C->g0[d] = g0[d];
        C->gamp[d] = gamp[d];
    }
    C->gomega = gomega;
    C->rho_out = rho_out;
    for (int64_t k = 0; k < nf; ++k)
        for (int i = 0; i < NQ; ++i) C->fpost[k * NQ + i] = weight(i);
    C->n = 0;
    stream(C);
    apply_open_boundaries(C, 0);
    return C;
}

/* Collision operator of the case: 0 CHM-MRT (default), 1 SRT with the second-order
 * equilibrium, 2 TRT with the second-order equilibrium and magic parameter `magic`. */
int oracle_set_collision(oracle_case* C, int model, double magic)
{
    if (model < 0 || model > 2 || !(magic > 0.0)) return 1;
    C->collision = model;
    C->magic = magic;
    return 0;
}

int oracle_set_waveform(oracle_case* C, const double* a, const double* b, int nh, double period,
                        double u_peak)
{
    if (nh < 0 || nh > 15 || !(period >= 1.0)) return -1;
    for (int k = 0; k <= nh; ++k) C->wa[k] = a[k];
    for (int k = 0; k < nh; ++k) C->wb[k] = b[k];
    C->wnh = nh;
    C->wP = period;
    C->wpeak = u_peak;
    C->has_wave = 1;
    apply_open_boundaries(C, C->n);
    return 0;
}

/* stream (pull form of the LBE) from fpost into f, with the wall rules on wall links */
static void stream(oracle_case* C)
{
    const int64_t nf = C->nfluid;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        int64_t b = C->cell[k];
        int x = (int)(b % C->nx), y = (int)((b / C->nx) % C->ny),
            z = (int)(b / ((int64_t)C->nx * C->ny));
        for (int i = 0; i < NQ; ++i) {
            int64_t src = shifted(C, x, y, z, i, -1);
            double v;
            if (src >= 0) {
                v = C->fpost[src * NQ + i];
            } else {
                /* wall link: unknown alpha = i, beta = opposite(i) points into the wall */
                int beta = opposite(i);
                double q = C->qlink[k * NQ + i];
                double fb = C->fpost[k * NQ + beta];
                if (q == 0.0) {
                    v = fb; /* halfway bounce-back */
                } else if (q < 0.5) {
                    /* Bouzidi, q < 1/2: needs f*_beta at x_f + c_alpha */
                    int64_t nb = shifted(C, x, y, z, i, +1);
                    v = (nb >= 0) ? 2.0 * q * fb + (1.0 - 2.0 * q) * C->fpost[nb * NQ + beta] : fb;
                } else {
                    v = fb / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * C->fpost[k * NQ + i];
                }
            }
            C->f[k * NQ + i] = v;
        }
    }
}

void oracle_step(oracle_case* C, int64_t nsteps)
{
    const int64_t nf = C->nfluid;
    for (int64_t s = 0; s < nsteps; ++s) {
        double g[3];
        gforce(C, C->n, g);
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k) {
            if (C->collision != 0) {
                const double tk = C->tau_cell ? C->tau_cell[k] : C->tau;
                if (C->collision == 1) oracle_collide_srt2(C->f + k * NQ, g, tk, C->fpost + k * NQ);
                else oracle_collide_trt2(C->f + k * NQ, g, tk, C->magic, C->fpost + k * NQ);
            } else if (C->tau_cell) {
                double sk[NQ];
                oracle_rates(C->tau_cell[k], C->omega_hi, sk);
                oracle_collide(C->f + k * NQ, g, sk, C->fpost + k * NQ);
            } else {
                oracle_collide(C->f + k * NQ, g, C->s, C->fpost + k * NQ);
            }
        }
        stream(C);
        C->n += 1;
        apply_open_boundaries(C, C->n);
    }
}

/* Initial condition from macroscopic fields on the dense box: the post-collision populations
 * of time level n-1 are set to the equilibrium f_eq(rho, u) of each fluid cell, then streamed
 * and closed at the current time level n.  The default state (rho = 1, u = 0) streams to w. */
void oracle_init_equilibrium(oracle_case* C, const double* rho, const double* u)
{
    int64_t nbox = (int64_t)C->nx * C->ny * C->nz;
    for (int64_t k = 0; k < C->nfluid; ++k) {
        int64_t b = C->cell[k];
        double uu[3] = {u[b], u[nbox + b], u[2 * nbox + b]};
        oracle_feq_product(rho[b], uu, C->fpost + k * NQ);
    }
    stream(C);
    apply_open_boundaries(C, C->n);
}

/* Velocity correction of the learned coarse-grid corrector (not in the paper): at every fluid
 * cell but inlet and outlet cells, with rho and u of level n (u with the half-force shift), the post-collision populations
 * of level n-1 gain f_eq(rho, u + du) - f_eq(rho, u); level n is then streamed and closed again.
 * du: three planes on the dense box. */
void oracle_apply_velocity_correction(oracle_case* C, const double* du)
{
    int64_t nbox = (int64_t)C->nx * C->ny * C->nz;
    double g[3];
    gforce(C, C->n, g);
    for (int64_t k = 0; k < C->nfluid; ++k) {
        if (C->kind[k] >= 2) continue; /* inlet/outlet closures rebuild their unknowns */
        const double* f = C->f + k * NQ;
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NQ; ++i) {
            r += f[i];
            for (int d = 0; d < 3; ++d) j[d] += cvel(i, d) * f[i];
        }
        int64_t b = C->cell[k];
        double u0[3], u1[3], fa[NQ], fb[NQ];
        for (int d = 0; d < 3; ++d) {
            u0[d] = j[d] / r + 0.5 * g[d];
            u1[d] = u0[d] + du[d * nbox + b];
        }
        oracle_feq_product(r, u1, fa);
        oracle_feq_product(r, u0, fb);
        for (int i = 0; i < NQ; ++i) C->fpost[k * NQ + i] += fa[i] - fb[i];
    }
    stream(C);
    apply_open_boundaries(C, C->n);
}

/* rho and u (with the half-force shift at the current time level) on the dense box, x fastest;
 * solid cells get rho = 0, u = 0. */
void oracle_macroscopic(const oracle_case* C, double* rho, double* u)
{
    int64_t nbox = (int64_t)C->nx * C->ny * C->nz;
    double g[3];
    gforce(C, C->n, g);
    for (int64_t b = 0; b < nbox; ++b) {
        rho[b] = 0.0;
        u[b] = u[nbox + b] = u[2 * nbox + b] = 0.0;
    }
    for (int64_t k = 0; k < C->nfluid; ++k) {
        const double* f = C->f + k * NQ;
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NQ; ++i) {
            r += f[i];
            for (int d = 0; d < 3; ++d) j[d] += cvel(i, d) * f[i];
        }
        int64_t b = C->cell[k];
        rho[b] = r;
        for (int d = 0; d < 3; ++d) u[d * nbox + b] = j[d] / r + 0.5 * g[d];
    }
}

int64_t oracle_nfluid(const oracle_case* C) { return C->nfluid; }
int64_t oracle_time(const oracle_case* C) { return C->n; }

/* populations f(x, n) of the fluid cells in increasing box order, [nfluid][27] */
void oracle_get_f(const oracle_case* C, double* out)
{
    memcpy(out, C->f, sizeof(double) * (size_t)C->nfluid * NQ);
}

void oracle_set_f(oracle_case* C, const double* in)
{
    memcpy(C->f, in, sizeof(double) * (size_t)C->nfluid * NQ);
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
