/*
 * FP64 CPU oracle for the per-pose protein-ligand docking energy (miniBUDE
 * "fasten", arxiv 2509.21039 Sec. 2.2, Listing 4; FLOP count Eq. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference the CUDA path is checked against.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, calls or falls back to it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (plain triple loop, in the order of Listing 4):
 *   for every pose k:    R_k = Rz(a2) * Ry(a1) * Rx(a0),  t_k = (t0, t1, t2)
 *     for every ligand atom l:     x' = R_k x_l + t_k
 *       for every protein atom p:  E_k += e(type_l, type_p, |x' - x_p|)
 *   energy[k] = 0.5 * E_k            (Listing 4 stores half the pose total)
 *
 * Pose layout: six arrays, angles a0..a2 then translations t0..t2, with the
 * first angle driving the rotation about x (Listing 4).  The first matrix
 * element is cos(a1)*cos(a2) as in Listing 4; the product Rz*Ry*Rx is the
 * reading that gives it (pinned by basis-vector tests).
 *
 * The paper describes fasten as scoring how strongly two molecules interact
 * (Sec. 2.2) but prints no forcefield, so the pair energy e(a, b, d) -- a
 * steric, an electrostatic and a desolvation term -- is this project's own
 * definition, built only from the per-type parameters radius r, hardness h,
 * charge-like q and hydrogen-bond class hb (0 none, 1 donor, 2 acceptor):
 *
 *   R = r_a + r_b          H = (h_a + h_b) / 2          Q = q_a * q_b
 *   w = 2 if {hb_a, hb_b} == {donor, acceptor} else 1
 *   S = K_D if exactly one of hb_a, hb_b is non-zero else 0
 *   s = d - R                                   surface separation
 *   phi(u) = 1 for u <= 0, (1-u)^2 (1+2u) for 0 < u < 1, 0 for u >= 1
 *   e = H (s/R)^2 [s < 0]  +  K_E Q w phi(s / D_E)  +  S phi(s / D_D)
 *   K_E = 4, D_E = 4 A, K_D = 0.5, D_D = 2 A
 *
 * Every term is zero for d >= R + 4 A, so that is the cutoff.  The pose
 * gradient follows from the chain rule through x' = R x + t (see
 * oracle_pose_grad).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define ORACLE_KE 4.0
#define ORACLE_DE 4.0
#define ORACLE_KD 0.5
#define ORACLE_DD 2.0

/* C1 cubic switch: 1 below 0, 0 above 1, smooth step in between. */
static double switch_phi(double u)
{
    if (u <= 0.0) return 1.0;
    if (u >= 1.0) return 0.0;
    return (1.0 - u) * (1.0 - u) * (1.0 + 2.0 * u);
}

/* d phi / d u: zero outside (0, 1), -6 u (1 - u) inside. */
static double switch_dphi(double u)
{
    if (u <= 0.0 || u >= 1.0) return 0.0;
    return -6.0 * u * (1.0 - u);
}

/* Type-pair parameters of the combination rules above. */
typedef struct {
    double R, H, QW, S;
} pair_params;

static pair_params combine(double ra, double ha, double qa, int hba,
                           double rb, double hb_, double qb, int hbb)
{
    pair_params p;
    p.R = ra + rb;
    p.H = 0.5 * (ha + hb_);
    double w = ((hba == 1 && hbb == 2) || (hba == 2 && hbb == 1)) ? 2.0 : 1.0;
    p.QW = ORACLE_KE * qa * qb * w;
    p.S = ((hba != 0) != (hbb != 0)) ? ORACLE_KD : 0.0;
    return p;
}

static double pair_energy_pp(const pair_params* p, double d)
{
    double s = d - p->R;
    double steric = (s < 0.0) ? p->H * (s / p->R) * (s / p->R) : 0.0;
    double elec = p->QW * switch_phi(s / ORACLE_DE);
    double desolv = p->S * switch_phi(s / ORACLE_DD);
    return steric + elec + desolv;
}

static double pair_denergy_pp(const pair_params* p, double d)
{
    double s = d - p->R;
    double steric = (s < 0.0) ? 2.0 * p->H * s / (p->R * p->R) : 0.0;
    double elec = p->QW * switch_dphi(s / ORACLE_DE) / ORACLE_DE;
    double desolv = p->S * switch_dphi(s / ORACLE_DD) / ORACLE_DD;
    return steric + elec + desolv;
}

/* e(a, b, d) for two atoms with explicit parameters. */
double oracle_pair_energy(double ra, double ha, double qa, int hba,
                          double rb, double hb_, double qb, int hbb, double d)
{
    pair_params p = combine(ra, ha, qa, hba, rb, hb_, qb, hbb);
    return pair_energy_pp(&p, d);
}

/* de/dd for two atoms with explicit parameters. */
double oracle_pair_denergy(double ra, double ha, double qa, int hba,
                           double rb, double hb_, double qb, int hbb, double d)
{
    pair_params p = combine(ra, ha, qa, hba, rb, hb_, qb, hbb);
    return pair_denergy_pp(&p, d);
}

static void matmul3(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = acc;
        }
}

static void rot_x(double a, double M[9])
{
    double c = cos(a), s = sin(a);
    double r[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    for (int i = 0; i < 9; ++i) M[i] = r[i];
}

static void rot_y(double a, double M[9])
{
    double c = cos(a), s = sin(a);
    double r[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    for (int i = 0; i < 9; ++i) M[i] = r[i];
}

static void rot_z(double a, double M[9])
{
    double c = cos(a), s = sin(a);
    double r[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    for (int i = 0; i < 9; ++i) M[i] = r[i];
}

/* Rotation of one pose: R = Rz(a2) Ry(a1) Rx(a0), row-major 3x3. */
void oracle_rotation(double a0, double a1, double a2, double R[9])
{
    double X[9], Y[9], Z[9], ZY[9];
    rot_x(a0, X);
    rot_y(a1, Y);
    rot_z(a2, Z);
    matmul3(Z, Y, ZY);
    matmul3(ZY, X, R);
}

typedef struct {
    int n_lig, n_pro, n_types;
    const double* lig_xyz;   /* [n_lig][3] */
    const int32_t* lig_type; /* [n_lig] */
    const double* pro_xyz;   /* [n_pro][3] */
    const int32_t* pro_type; /* [n_pro] */
    const double* radius;    /* [n_types] */
    const double* hardness;  /* [n_types] */
    const double* elsc;      /* [n_types] */
    const int32_t* hbtype;   /* [n_types] */
} oracle_deck;

static int check_deck(const oracle_deck* D)
{
    if (D->n_lig < 0 || D->n_pro < 0 || D->n_types < 0) return -1;
    for (int l = 0; l < D->n_lig; ++l)
        if (D->lig_type[l] < 0 || D->lig_type[l] >= D->n_types) return -1;
    for (int p = 0; p < D->n_pro; ++p)
        if (D->pro_type[p] < 0 || D->pro_type[p] >= D->n_types) return -1;
    return 0;
}

static pair_params deck_pair(const oracle_deck* D, int a, int b)
{
    return combine(D->radius[a], D->hardness[a], D->elsc[a], D->hbtype[a],
                   D->radius[b], D->hardness[b], D->elsc[b], D->hbtype[b]);
}

/*
 * Energy of poses [k0, k1).  poses is [6][n_poses].  energy[k] receives
 * 0.5 * sum_l sum_p e and, when abs_sum is not NULL, abs_sum[k] receives
 * 0.5 * sum_l sum_p |e| (the scale used for scaled-error comparisons).
 */
static void energies_range(const oracle_deck* D, int64_t n_poses,
                           const double* poses, int64_t k0, int64_t k1,
                           double* energy, double* abs_sum)
{
    for (int64_t k = k0; k < k1; ++k) {
        double R[9];
        oracle_rotation(poses[0 * n_poses + k], poses[1 * n_poses + k],
                        poses[2 * n_poses + k], R);
        double t[3] = {poses[3 * n_poses + k], poses[4 * n_poses + k],
                       poses[5 * n_poses + k]};
        double E = 0.0, A = 0.0;
        for (int l = 0; l < D->n_lig; ++l) {
            const double* x = D->lig_xyz + 3 * l;
            double xp[3];
            for (int i = 0; i < 3; ++i)
                xp[i] = R[3 * i + 0] * x[0] + R[3 * i + 1] * x[1] +
                        R[3 * i + 2] * x[2] + t[i];
            for (int p = 0; p < D->n_pro; ++p) {
                const double* y = D->pro_xyz + 3 * p;
                double dx = xp[0] - y[0], dy = xp[1] - y[1], dz = xp[2] - y[2];
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                pair_params pp = deck_pair(D, D->lig_type[l], D->pro_type[p]);
                double e = pair_energy_pp(&pp, d);
                E += e;
                A += fabs(e);
            }
        }
        energy[k] = 0.5 * E;
        if (abs_sum) abs_sum[k] = 0.5 * A;
    }
}

int oracle_energies(int n_lig, const double* lig_xyz, const int32_t* lig_type,
                    int n_pro, const double* pro_xyz, const int32_t* pro_type,
                    int n_types, const double* radius, const double* hardness,
                    const double* elsc, const int32_t* hbtype,
                    int64_t n_poses, const double* poses, double* energy,
                    double* abs_sum, int n_threads)
{
    oracle_deck D = {n_lig, n_pro, n_types, lig_xyz, lig_type, pro_xyz,
                     pro_type, radius, hardness, elsc, hbtype};
    if (n_poses < 0 || check_deck(&D) != 0) return -1;
#ifdef _OPENMP
    if (n_threads > 0) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
        for (int64_t k = 0; k < n_poses; ++k)
            energies_range(&D, n_poses, poses, k, k + 1, energy, abs_sum);
        return 0;
    }
#endif
    (void)n_threads;
    energies_range(&D, n_poses, poses, 0, n_poses, energy, abs_sum);
    return 0;
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Gradient of energy[k] with respect to the six pose parameters.
 *
 * With g_l = dE/dx'_l = 0.5 * sum_p e'(d) (x'_l - x_p) / d and
 * r_l = x'_l - t = R x_l:
 *   dE/dt      = F   = sum_l g_l
 *   dE/da_j    = sum_l g_l . (dR/da_j x_l)
 * dR/da_j x_l is written out from the product R = Rz Ry Rx by differentiating
 * the factor that holds a_j, e.g. dR/da1 = Rz Ry' Rx, so no torque identity is
 * assumed here.  A pair at d = 0 contributes no gradient (direction
 * undefined, and e'(0) (x'-p)/d has no limit).  When scale is not NULL it
 * receives, per pose, 0.5 sum |e'| |r_l| (a bound on each angle derivative)
 * and 0.5 sum |e'| (a bound on each translation derivative): [2][n_poses].
 */
static void grad_range(const oracle_deck* D, int64_t n_poses,
                       const double* poses, int64_t k0, int64_t k1,
                       double* energy, double* grad, double* scale)
{
    for (int64_t k = k0; k < k1; ++k) {
        double a0 = poses[0 * n_poses + k], a1 = poses[1 * n_poses + k],
               a2 = poses[2 * n_poses + k];
        double X[9], Y[9], Z[9], dX[9], dY[9], dZ[9];
        rot_x(a0, X);
        rot_y(a1, Y);
        rot_z(a2, Z);
        /* derivatives of the elementary rotations */
        double c0 = cos(a0), s0 = sin(a0), c1 = cos(a1), s1 = sin(a1),
               c2 = cos(a2), s2 = sin(a2);
        double dx_[9] = {0, 0, 0, 0, -s0, -c0, 0, c0, -s0};
        double dy_[9] = {-s1, 0, c1, 0, 0, 0, -c1, 0, -s1};
        double dz_[9] = {-s2, -c2, 0, c2, -s2, 0, 0, 0, 0};
        for (int i = 0; i < 9; ++i) {
            dX[i] = dx_[i];
            dY[i] = dy_[i];
            dZ[i] = dz_[i];
        }
        double T[9], R[9], D0[9], D1[9], D2[9];
        matmul3(Z, Y, T);
        matmul3(T, X, R);
        matmul3(T, dX, D0); /* Rz Ry Rx' */
        matmul3(Z, dY, T);
        matmul3(T, X, D1); /* Rz Ry' Rx */
        matmul3(dZ, Y, T);
        matmul3(T, X, D2); /* Rz' Ry Rx */
        double t[3] = {poses[3 * n_poses + k], poses[4 * n_poses + k],
                       poses[5 * n_poses + k]};
        double E = 0.0, G[6] = {0, 0, 0, 0, 0, 0};
        double abs_f = 0.0, abs_t = 0.0; /* error scales: sum |e'|, sum |r| |e'| */
        for (int l = 0; l < D->n_lig; ++l) {
            const double* x = D->lig_xyz + 3 * l;
            double xp[3];
            for (int i = 0; i < 3; ++i)
                xp[i] = R[3 * i + 0] * x[0] + R[3 * i + 1] * x[1] +
                        R[3 * i + 2] * x[2] + t[i];
            double g[3] = {0, 0, 0}, abs_l = 0.0;
            for (int p = 0; p < D->n_pro; ++p) {
                const double* y = D->pro_xyz + 3 * p;
                double dv[3] = {xp[0] - y[0], xp[1] - y[1], xp[2] - y[2]};
                double d = sqrt(dot3(dv, dv));
                pair_params pp = deck_pair(D, D->lig_type[l], D->pro_type[p]);
                E += pair_energy_pp(&pp, d);
                if (d > 0.0) {
                    double de = pair_denergy_pp(&pp, d);
                    double f = de / d;
                    for (int i = 0; i < 3; ++i) g[i] += f * dv[i];
                    abs_l += fabs(de);
                }
            }
            double r[3] = {xp[0] - t[0], xp[1] - t[1], xp[2] - t[2]};
            abs_f += abs_l;
            abs_t += abs_l * sqrt(dot3(r, r));
            /* 0.5 factor of the output applied once at the end */
            double v0[3], v1[3], v2[3];
            for (int i = 0; i < 3; ++i) {
                v0[i] = D0[3 * i] * x[0] + D0[3 * i + 1] * x[1] + D0[3 * i + 2] * x[2];
                v1[i] = D1[3 * i] * x[0] + D1[3 * i + 1] * x[1] + D1[3 * i + 2] * x[2];
                v2[i] = D2[3 * i] * x[0] + D2[3 * i + 1] * x[1] + D2[3 * i + 2] * x[2];
            }
            G[0] += dot3(g, v0);
            G[1] += dot3(g, v1);
            G[2] += dot3(g, v2);
            G[3] += g[0];
            G[4] += g[1];
            G[5] += g[2];
        }
        if (energy) energy[k] = 0.5 * E;
        for (int j = 0; j < 6; ++j) grad[j * n_poses + k] = 0.5 * G[j];
        if (scale) {
            scale[k] = 0.5 * abs_t;           /* bounds |dE/da_j| */
            scale[n_poses + k] = 0.5 * abs_f; /* bounds |dE/dt_j| */
        }
    }
}

int oracle_pose_grad(int n_lig, const double* lig_xyz, const int32_t* lig_type,
                     int n_pro, const double* pro_xyz, const int32_t* pro_type,
                     int n_types, const double* radius, const double* hardness,
                     const double* elsc, const int32_t* hbtype,
                     int64_t n_poses, const double* poses, double* energy,
                     double* grad, double* scale, int n_threads)
{
    oracle_deck D = {n_lig, n_pro, n_types, lig_xyz, lig_type, pro_xyz,
                     pro_type, radius, hardness, elsc, hbtype};
    if (n_poses < 0 || check_deck(&D) != 0) return -1;
#ifdef _OPENMP
    if (n_threads > 0) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
        for (int64_t k = 0; k < n_poses; ++k)
            grad_range(&D, n_poses, poses, k, k + 1, energy, grad, scale);
        return 0;
    }
#endif
    (void)n_threads;
    grad_range(&D, n_poses, poses, 0, n_poses, energy, grad, scale);
    return 0;
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}


/*
 * Gradient of L = sum_k w_k energy[k] with respect to the ligand atom
 * coordinates (in the ligand frame, before the pose) and to the per-type
 * forcefield parameters radius, hardness and elsc.
 *
 *   dL/dx_l  = sum_k w_k 0.5 sum_p R_k^T e'(d) (x'_l - x_p) / d
 * and, for a pair of types a (ligand) and b (protein), from the
 * combination rules R = r_a + r_b, H = (h_a + h_b)/2, Q = q_a q_b:
 *   de/dr_a = de/dr_b = de/dR
 *   de/dh_a = de/dh_b = (1/2) de/dH
 *   de/dq_a = K_E w q_b phi(s/D_E),  de/dq_b = K_E w q_a phi(s/D_E)
 * with de/dR = -2 H (s/R) d / R^2 [s<0] - QW phi'(s/D_E)/D_E
 *              - S phi'(s/D_D)/D_D  and  de/dH = (s/R)^2 [s<0].
 * lig_grad is [n_lig][3], ff_grad is [n_types][3] (radius, hardness, elsc);
 * weights may be NULL (all ones).  A pair at d = 0 adds nothing to lig_grad.
 */
int oracle_param_grad(int n_lig, const double* lig_xyz, const int32_t* lig_type,
                      int n_pro, const double* pro_xyz, const int32_t* pro_type,
                      int n_types, const double* radius, const double* hardness,
                      const double* elsc, const int32_t* hbtype,
                      int64_t n_poses, const double* poses, const double* weights,
                      double* lig_grad, double* ff_grad)
{
    oracle_deck D = {n_lig, n_pro, n_types, lig_xyz, lig_type, pro_xyz,
                     pro_type, radius, hardness, elsc, hbtype};
    if (n_poses < 0 || check_deck(&D) != 0) return -1;
    for (int i = 0; i < 3 * n_lig; ++i) lig_grad[i] = 0.0;
    for (int i = 0; i < 3 * n_types; ++i) ff_grad[i] = 0.0;
    for (int64_t k = 0; k < n_poses; ++k) {
        double wk = weights ? weights[k] : 1.0;
        double R[9];
        oracle_rotation(poses[0 * n_poses + k], poses[1 * n_poses + k],
                        poses[2 * n_poses + k], R);
        double t[3] = {poses[3 * n_poses + k], poses[4 * n_poses + k],
                       poses[5 * n_poses + k]};
        for (int l = 0; l < n_lig; ++l) {
            const double* x = lig_xyz + 3 * l;
            double xp[3];
            for (int i = 0; i < 3; ++i)
                xp[i] = R[3 * i + 0] * x[0] + R[3 * i + 1] * x[1] +
                        R[3 * i + 2] * x[2] + t[i];
            int a = lig_type[l];
            double g[3] = {0, 0, 0};
            for (int p = 0; p < n_pro; ++p) {
                int b = pro_type[p];
                const double* y = pro_xyz + 3 * p;
                double dv[3] = {xp[0] - y[0], xp[1] - y[1], xp[2] - y[2]};
                double d = sqrt(dot3(dv, dv));
                pair_params pp = deck_pair(&D, a, b);
                double s = d - pp.R;
                double dR = -pp.QW * switch_dphi(s / ORACLE_DE) / ORACLE_DE -
                            pp.S * switch_dphi(s / ORACLE_DD) / ORACLE_DD;
                double dH = 0.0;
                if (s < 0.0) {
                    dR += -2.0 * pp.H * (s / pp.R) * d / (pp.R * pp.R);
                    dH = (s / pp.R) * (s / pp.R);
                }
                double wab = ((hbtype[a] == 1 && hbtype[b] == 2) ||
                              (hbtype[a] == 2 && hbtype[b] == 1)) ? 2.0 : 1.0;
                double phiE = switch_phi(s / ORACLE_DE);
                double f = 0.5 * wk;
                ff_grad[3 * a + 0] += f * dR;
                ff_grad[3 * b + 0] += f * dR;
                ff_grad[3 * a + 1] += f * 0.5 * dH;
                ff_grad[3 * b + 1] += f * 0.5 * dH;
                ff_grad[3 * a + 2] += f * ORACLE_KE * wab * elsc[b] * phiE;
                ff_grad[3 * b + 2] += f * ORACLE_KE * wab * elsc[a] * phiE;
                if (d > 0.0) {
                    double c = pair_denergy_pp(&pp, d) / d;
                    for (int i = 0; i < 3; ++i) g[i] += c * dv[i];
                }
            }
            /* dL/dx_l += w_k 0.5 R^T g */
            for (int j = 0; j < 3; ++j)
                lig_grad[3 * l + j] += 0.5 * wk *
                    (R[0 * 3 + j] * g[0] + R[1 * 3 + j] * g[1] + R[2 * 3 + j] * g[2]);
        }
    }
    return 0;
}

/*
 * Parity scales of oracle_param_grad: every output element is a sum of
 * terms, one per (pose, ligand atom, protein atom[, component]); each scale
 * element is the same sum with every term replaced by its absolute value,
 * and the three parts of de/dR and of de/dd (steric, electrostatic,
 * desolvation) taken as separate terms.  The rounding error of a computed
 * sum is bounded by a small multiple of the unit roundoff times this sum of
 * absolute values (the standard bound for recursive summation), so it is
 * the scale against which a lower-precision result of the same sum is
 * judged element by element.  Same arguments as oracle_param_grad;
 * lig_scale is [n_lig][3], ff_scale [n_types][3].
 */
int oracle_param_grad_scale(int n_lig, const double* lig_xyz, const int32_t* lig_type,
                            int n_pro, const double* pro_xyz, const int32_t* pro_type,
                            int n_types, const double* radius, const double* hardness,
                            const double* elsc, const int32_t* hbtype,
                            int64_t n_poses, const double* poses, const double* weights,
                            double* lig_scale, double* ff_scale)
{
    oracle_deck D = {n_lig, n_pro, n_types, lig_xyz, lig_type, pro_xyz,
                     pro_type, radius, hardness, elsc, hbtype};
    if (n_poses < 0 || check_deck(&D) != 0) return -1;
    for (int i = 0; i < 3 * n_lig; ++i) lig_scale[i] = 0.0;
    for (int i = 0; i < 3 * n_types; ++i) ff_scale[i] = 0.0;
    for (int64_t k = 0; k < n_poses; ++k) {
        double wk = fabs(weights ? weights[k] : 1.0);
        double R[9];
        oracle_rotation(poses[0 * n_poses + k], poses[1 * n_poses + k],
                        poses[2 * n_poses + k], R);
        double t[3] = {poses[3 * n_poses + k], poses[4 * n_poses + k],
                       poses[5 * n_poses + k]};
        for (int l = 0; l < n_lig; ++l) {
            const double* x = lig_xyz + 3 * l;
            double xp[3];
            for (int i = 0; i < 3; ++i)
                xp[i] = R[3 * i + 0] * x[0] + R[3 * i + 1] * x[1] +
                        R[3 * i + 2] * x[2] + t[i];
            int a = lig_type[l];
            for (int p = 0; p < n_pro; ++p) {
                int b = pro_type[p];
                const double* y = pro_xyz + 3 * p;
                double dv[3] = {xp[0] - y[0], xp[1] - y[1], xp[2] - y[2]};
                double d = sqrt(dot3(dv, dv));
                pair_params pp = deck_pair(&D, a, b);
                double s = d - pp.R;
                /* the parts of de/dd, each as an absolute value */
                double e_el = fabs(pp.QW * switch_dphi(s / ORACLE_DE) / ORACLE_DE);
                double e_de = fabs(pp.S * switch_dphi(s / ORACLE_DD) / ORACLE_DD);
                double e_st = 0.0, r_st = 0.0, dH = 0.0;
                if (s < 0.0) {
                    e_st = fabs(2.0 * pp.H * s / (pp.R * pp.R));
                    r_st = fabs(2.0 * pp.H * (s / pp.R) * d / (pp.R * pp.R));
                    dH = (s / pp.R) * (s / pp.R);
                }
                double wab = ((hbtype[a] == 1 && hbtype[b] == 2) ||
                              (hbtype[a] == 2 && hbtype[b] == 1)) ? 2.0 : 1.0;
                double phiE = switch_phi(s / ORACLE_DE);
                double f = 0.5 * wk;
                double r_abs = r_st + e_el + e_de;
                ff_scale[3 * a + 0] += f * r_abs;
                ff_scale[3 * b + 0] += f * r_abs;
                ff_scale[3 * a + 1] += f * 0.5 * dH;
                ff_scale[3 * b + 1] += f * 0.5 * dH;
                ff_scale[3 * a + 2] += f * ORACLE_KE * wab * fabs(elsc[b]) * phiE;
                ff_scale[3 * b + 2] += f * ORACLE_KE * wab * fabs(elsc[a]) * phiE;
                if (d > 0.0) {
                    double c = (e_st + e_el + e_de) / d;
                    for (int j = 0; j < 3; ++j)
                        for (int i = 0; i < 3; ++i)
                            lig_scale[3 * l + j] += f * fabs(R[3 * i + j]) * c * fabs(dv[i]);
                }
            }
        }
    }
    return 0;
}
