/*
 * FP64 CPU oracle for the two-electron part of the Hartree-Fock Fock matrix
 * over s-type Gaussian basis functions (arxiv 2509.21039, Sec. 2.2,
 * Listing 5; Table 4) -- TEST INFRASTRUCTURE ONLY, used by the test suite
 * and never by the product library.
 *
 * Each atom i carries one contracted s function
 *   phi_i(r) = sum_a c_a N(x_a) exp(-x_a |r - R_i|^2),  N(x) = (2x/pi)^(3/4),
 * with the same exponents x_a and coefficients c_a on every atom.  For
 * primitives a, b, c, d on centres A, B, C, D (p = x_a + x_b, q = x_c + x_d,
 * P = (x_a A + x_b B)/p, Q likewise, rho = p q / (p + q)):
 *   (ab|cd) = N_a N_b N_c N_d 2 pi^(5/2) / (p q sqrt(p + q))
 *             exp(-x_a x_b |A-B|^2 / p) exp(-x_c x_d |C-D|^2 / q) F0(rho |P-Q|^2)
 * with the Boys function F0(t) = (1/2) sqrt(pi/t) erf(sqrt t), F0(0) = 1.
 * The contracted integral (ij|kl) sums c_a c_b c_c c_d (ab|cd) over all
 * primitive quartets.  The Fock contribution of density D is the plain sum
 *   G_ij = sum_kl D_kl [ 2 (ij|kl) - (ik|jl) ].
 */
#include <math.h>
#include <stdint.h>

static const double HF_PI = 3.14159265358979323846;

/* Boys function of order 0, from its erf closed form (series near 0). */
double oracle_boys0(double t)
{
    if (t < 1e-10) return 1.0 - t / 3.0;
    double st = sqrt(t);
    return 0.5 * sqrt(HF_PI / t) * erf(st);
}

/* Normalised primitive integral (ab|cd). */
double oracle_prim_eri(double xa, const double* A, double xb, const double* B,
                       double xc, const double* C, double xd, const double* D)
{
    double p = xa + xb, q = xc + xd;
    double AB2 = 0, CD2 = 0, PQ2 = 0;
    for (int k = 0; k < 3; ++k) {
        double ab = A[k] - B[k], cd = C[k] - D[k];
        AB2 += ab * ab;
        CD2 += cd * cd;
        double P = (xa * A[k] + xb * B[k]) / p;
        double Q = (xc * C[k] + xd * D[k]) / q;
        PQ2 += (P - Q) * (P - Q);
    }
    double na = pow(2.0 * xa / HF_PI, 0.75), nb = pow(2.0 * xb / HF_PI, 0.75);
    double nc = pow(2.0 * xc / HF_PI, 0.75), nd = pow(2.0 * xd / HF_PI, 0.75);
    double rho = p * q / (p + q);
    return na * nb * nc * nd * 2.0 * pow(HF_PI, 2.5) / (p * q * sqrt(p + q)) *
           exp(-xa * xb * AB2 / p) * exp(-xc * xd * CD2 / q) * oracle_boys0(rho * PQ2);
}

/* Contracted (ij|kl) for centres A, B, C, D. */
double oracle_eri(int ng, const double* xpnt, const double* coef, const double* A,
                  const double* B, const double* C, const double* D)
{
    double s = 0.0;
    for (int a = 0; a < ng; ++a)
        for (int b = 0; b < ng; ++b)
            for (int c = 0; c < ng; ++c)
                for (int d = 0; d < ng; ++d)
                    s += coef[a] * coef[b] * coef[c] * coef[d] *
                         oracle_prim_eri(xpnt[a], A, xpnt[b], B, xpnt[c], C, xpnt[d], D);
    return s;
}

/*
 * G_ij for the listed entries (rows[e], cols[e]), e < n_entries, by the plain
 * sum over all k, l.  geom is [n][3], dens [n][n] row-major.
 */
void oracle_hf_fock_entries(int n, const double* geom, int ng, const double* xpnt,
                            const double* coef, const double* dens, int n_entries,
                            const int32_t* rows, const int32_t* cols, double* out)
{
    for (int e = 0; e < n_entries; ++e) {
        int i = rows[e], j = cols[e];
        double g = 0.0;
        for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l) {
                double J = oracle_eri(ng, xpnt, coef, geom + 3 * i, geom + 3 * j,
                                      geom + 3 * k, geom + 3 * l);
                double K = oracle_eri(ng, xpnt, coef, geom + 3 * i, geom + 3 * k,
                                      geom + 3 * j, geom + 3 * l);
                g += dens[k * n + l] * (2.0 * J - K);
            }
        out[e] = g;
    }
}

/*
 * Parity scale of G_ij: the plain sum above with every term replaced by its
 * absolute value, S_ij = sum_kl |D_kl| (2 |(ij|kl)| + |(ik|jl)|).  The
 * rounding error of any evaluation of G_ij as a sum of these terms is
 * bounded by a small multiple of the unit roundoff times S_ij.
 */
void oracle_hf_fock_scale_entries(int n, const double* geom, int ng, const double* xpnt,
                                  const double* coef, const double* dens, int n_entries,
                                  const int32_t* rows, const int32_t* cols, double* out)
{
    for (int e = 0; e < n_entries; ++e) {
        int i = rows[e], j = cols[e];
        double g = 0.0;
        for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l) {
                double J = oracle_eri(ng, xpnt, coef, geom + 3 * i, geom + 3 * j,
                                      geom + 3 * k, geom + 3 * l);
                double K = oracle_eri(ng, xpnt, coef, geom + 3 * i, geom + 3 * k,
                                      geom + 3 * j, geom + 3 * l);
                g += fabs(dens[k * n + l]) * (2.0 * fabs(J) + fabs(K));
            }
        out[e] = g;
    }
}
