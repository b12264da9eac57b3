/*
 * sdm_oracle.c -- plain, slow, single-threaded FP64 reference of the
 * Super-Droplet Method (SDM) coalescence step (Bartman & Arabas,
 * arXiv:2101.06318).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may link, load or call this file; only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
 * header, table or constant generator with the CUDA path: every constant and
 * table below is written out here from the definitions in the method
 * description, and the CUDA sources carry their own copy.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fno-fast-math -shared -fPIC
 *        (FMA contraction off: every FP64 operation is rounded separately, in
 *        the order written.)
 *
 * What each function follows:
 *   philox4x32_10      Salmon et al., SC'11 "Parallel random numbers: as easy
 *                      as 1, 2, 3" (counter-based RNG); project RNG contract
 *                      (which counter words mean what) is stated below.
 *   sdmo_step          Sec. 3.2, Fig. "fig:algo" (Step 0..3 in that order);
 *                      Sec. 2.2 Steps 1-3; eq. (p); gamma = ceil(p - phi);
 *                      eq. (gamma2); eqs. (coal_attr_0) and (coal) (cases 1/2);
 *                      the paper's listing of the Numba update routine (tie
 *                      rule, g == 0 skip, case-2 attribute expression).
 *   golovin kernel     Sec. 4, a(v1, v2) = b (v1 + v2).
 *   electric field     Sec. 4 names a parametric kernel for electric-field
 *                      effects without a formula: project definition below
 *                      (sdmo_efficiency_field), parity unpinned against physics.
 *   gravitational      Sec. 4 names a "gravitational kernel with parametric
 *                      terminal velocity" but gives no formula; the project
 *                      definition used here is pi (r1+r2)^2 |vt1 - vt2| E(r1,r2)
 *                      with a three-regime power-law vt and a tabulated,
 *                      bilinearly interpolated efficiency E (parity unpinned
 *                      against physics: the paper's comparison data are absent).
 *   spectrum           Sec. 4: mass per unit ln r, rho = 1000 kg/m^3 (in
 *                      __init__.py: per bin the exact sum of the terms xi v,
 *                      rounded once, by math.fsum).
 *   golovin_phi, i1e   Sec. 4, analytic Golovin solution (eq. 36 of Golovin
 *                      1963 as restated in the paper); I1e written from the
 *                      power series of I1 and the large-argument expansion
 *                      (Abramowitz & Stegun 9.7.1).
 *
 * RNG contract (project-defined; the paper only says "random permutation" and
 * phi ~ U[0,1)).  i is the position of an SD in its cell's list L_c (the live
 * SDs in slot order, Step 0), n = |L_c|:
 *   key = (seed & 0xffffffff, seed >> 32)
 *   phi of candidate pair m of cell c at step s:
 *       x = philox(ctr = (m >> 1, c, s, 1)); w = 2 (m & 1)
 *       u53 = ((x[w] << 32) | x[w+1]) >> 11 ;  phi = u53 * 2^-53
 *   Two shuffles (Step 1) are defined; the shuffled list is L'_c:
 *   SORT: shuffle key of position i = philox(ctr = (i >> 2, c, s, 0))[i & 3];
 *         L'_c = L_c sorted ascending by (key, i)       (the paper's GPU way).
 *   PRP:  cells with n <= 256 are shuffled exactly as by SORT; for n > 256,
 *         L'_c[q] = L_c[P(q)] with P a keyed bijection of [0, n): an
 *         eight-round alternating Feistel network on Z_A x Z_B (x = L B + R;
 *         A B = n with halves of floor(k/2) and k - floor(k/2) bits when
 *         n = 2^k, else A = ceil(sqrt n), B = ceil(n / A)), round function
 *         h = lowbias32(v ^ K_r) without its last step x ^= x >> 16 (C. Wellons'
 *         32-bit integer hash) of the other half v, added as floor(h M / 2^32)
 *         modulo the half's size M, round keys
 *         K_0..K_3 = philox(0, c, s, 2), K_4..K_7 = philox(1, c, s, 2), and
 *         cycle-walking (apply the network again while the value is >= n) to
 *         stay inside [0, n); A B < n + A makes walking rare.  (Below ~256 elements a Feistel network of this
 *         depth is measurably non-uniform; above, the pairings it produces
 *         pass the uniformity tests.)
 *   Pair m is (L'_c[2m], L'_c[2m+1]), m < floor(n/2).
 *
 * Slot model: SD storage is a fixed array of slots grouped by cell
 * (cell c owns slots [cell_start[c], cell_start[c+1])).  A slot with xi = 0 is
 * a removed SD.  After every step each cell is compacted stably: its live SDs
 * move, in order, to the front of its slots and the freed slots are set to
 * xi = 0 with all attributes 0 (the paper's Index shrink, Step 0 of the next
 * step).  Positions in L_c, not slots, identify SDs for the RNG, so the
 * results do not depend on this storage convention.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define SDMO_OK 0
#define SDMO_EINVAL 1
#define SDMO_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds, multipliers and Weyl key increments.    */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void sdmo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    int r;
    philox_round(c, k);
    for (r = 1; r < 10; ++r) {
        k[0] += PHILOX_W0;
        k[1] += PHILOX_W1;
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

uint32_t sdmo_shuffle_key(uint64_t seed, uint32_t cell, uint32_t step, uint32_t l)
{
    uint32_t key[2], ctr[4], x[4];
    seed_key(seed, key);
    ctr[0] = l >> 2; ctr[1] = cell; ctr[2] = step; ctr[3] = 0;
    sdmo_philox4x32_10(ctr, key, x);
    return x[l & 3];
}

/* The Feistel round function: lowbias32 (C. Wellons, "Prospecting for hash functions",
 * 2018) without its last step x ^= x >> 16.  A round uses floor(h M / 2^32) with M < 2^16,
 * which the top bits of h decide (alone when M is a power of two); that last step leaves the
 * top 16 bits unchanged. */
static uint32_t round_hash(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    return x;
}

#define SDMO_PRP_ROUNDS 8
#define SDMO_PRP_MIN_N 257   /* smaller cells are sorted by key */

/* Round keys of the PRP shuffle of cell c at step s. */
void sdmo_prp_keys(uint64_t seed, uint32_t cell, uint32_t step, uint32_t K[SDMO_PRP_ROUNDS])
{
    uint32_t key[2], ctr[4];
    seed_key(seed, key);
    ctr[0] = 0; ctr[1] = cell; ctr[2] = step; ctr[3] = 2;
    sdmo_philox4x32_10(ctr, key, K);
    ctr[0] = 1;
    sdmo_philox4x32_10(ctr, key, K + 4);
}

static uint32_t ceil_log2_u32(uint32_t n)
{
    uint32_t k = 0;
    while (k < 32 && (1ull << k) < (uint64_t)n) ++k;
    return k;
}

/* The network's domain for a list of n elements: x = L * B + R with L < A, R < B.
 *   n a power of two, n = 2^k: A = 2^floor(k/2), B = 2^(k - floor(k/2)) (so A B = n);
 *   otherwise: A = ceil(sqrt(n)), B = ceil(n / A) (so n <= A B < n + A). */
static void prp_domain(uint32_t n, uint32_t* A, uint32_t* B)
{
    if (n != 0 && (n & (n - 1)) == 0) {
        uint32_t k = ceil_log2_u32(n), a = k >> 1;
        *A = 1u << a;
        *B = 1u << (k - a);
        return;
    }
    uint32_t a = 1;
    while ((uint64_t)a * a < n) ++a;
    *A = a;
    *B = (n + a - 1) / a;
}

/* One pass of the alternating Feistel network on Z_A x Z_B: for r = 0..7, with
 * h = round_hash(v ^ K_r) of the other half v,
 *   even r: L = (L + floor(h A / 2^32)) mod A;   odd r: R = (R + floor(h B / 2^32)) mod B.
 * Each round is a bijection of Z_A x Z_B (it shifts one half by an amount that depends only on
 * the other half), so the pass is one too. */
static uint32_t feistel(uint32_t q, uint32_t A, uint32_t B, const uint32_t K[SDMO_PRP_ROUNDS])
{
    uint32_t L = q / B, R = q % B;
    int r;
    for (r = 0; r < SDMO_PRP_ROUNDS; ++r) {
        if ((r & 1) == 0) {
            const uint32_t h = round_hash(R ^ K[r]);
            L = (uint32_t)((L + (((uint64_t)h * A) >> 32)) % A);
        } else {
            const uint32_t h = round_hash(L ^ K[r]);
            R = (uint32_t)((R + (((uint64_t)h * B) >> 32)) % B);
        }
    }
    return L * B + R;
}

/* P(q): the keyed bijection of [0, n) (cycle-walking on [0, A B)). */
uint32_t sdmo_prp(uint32_t q, uint32_t n, const uint32_t K[SDMO_PRP_ROUNDS])
{
    uint32_t A, B;
    prp_domain(n, &A, &B);
    uint32_t e = feistel(q, A, B, K);
    while (e >= n) e = feistel(e, A, B, K);
    return e;
}

/* The whole permutation: out[q] = P(q) for q < n (a loop over sdmo_prp, for tests at large n). */
void sdmo_prp_perm(uint32_t n, const uint32_t K[SDMO_PRP_ROUNDS], uint32_t* out)
{
    uint32_t q;
    for (q = 0; q < n; ++q) out[q] = sdmo_prp(q, n, K);
}

uint64_t sdmo_phi_u53(uint64_t seed, uint32_t cell, uint32_t step, uint32_t m)
{
    uint32_t key[2], ctr[4], x[4];
    unsigned w = 2u * (m & 1u);
    seed_key(seed, key);
    ctr[0] = m >> 1; ctr[1] = cell; ctr[2] = step; ctr[3] = 1;
    sdmo_philox4x32_10(ctr, key, x);
    return ((((uint64_t)x[w]) << 32) | (uint64_t)x[w + 1]) >> 11;
}

double sdmo_phi(uint64_t seed, uint32_t cell, uint32_t step, uint32_t m)
{
    /* u53 < 2^53 converts exactly; the scaling by 2^-53 is exact. */
    return (double)sdmo_phi_u53(seed, cell, step, m) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Coalescence kernels a(v1, v2).                                            */
/* ------------------------------------------------------------------------ */
#define KERNEL_GOLOVIN 0
#define KERNEL_GRAVITATIONAL 1
#define KERNEL_ELECTRIC 2

/* Golovin additive kernel, Sec. 4: a = b (v1 + v2). */
double sdmo_kernel_golovin(double v1, double v2, double b)
{
    double s = v1 + v2;
    return b * s;
}

/* Cube root from + and * only (reproducible bit for bit, and no division,
 * which is slow in FP64 on some hardware): write x = m 2^e with m in [0.5, 1)
 * and e = 3q + rmd; seed y ~ m^(-1/3) with the quadratic
 * (0.456419 m - 1.19161) m + 1.73758 times 2^(-rmd/3); with M = m 2^rmd take
 * three Newton steps for the reciprocal cube root, y <- y + y (1 - M y^3)/3;
 * c = (M y) y ~ M^(1/3); one residual correction c <- c - (c^3 - M) y^2/3;
 * result c 2^q.  Within 1 ulp of libm's cbrt over the tested range.  Defined
 * for positive normal x. */
static uint64_t dbits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double bitsd(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

double sdmo_cbrt(double x)
{
    uint64_t u = dbits(x);
    int e = (int)((u >> 52) & 0x7ff) - 1022;          /* x = m 2^e, m in [0.5,1) */
    double m = bitsd((u & 0x800fffffffffffffull) | (1022ull << 52));
    const double two_m13[3] = {1.0, 0.7937005259840998, 0.6299605249474366};   /* 2^(-rmd/3) */
    const double third = 0.3333333333333333;
    int q, rmd, i;
    double y, M, c, r, t;
    q = (e >= 0) ? e / 3 : -((-e + 2) / 3);             /* floor(e / 3) */
    rmd = e - 3 * q;                                     /* 0, 1 or 2 */
    y = 0.456419 * m;
    y = y - 1.19161;
    y = y * m;
    y = y + 1.73758;
    y = y * two_m13[rmd];
    M = m;
    if (rmd == 1) M = m * 2.0;
    else if (rmd == 2) M = m * 4.0;                      /* M in [0.5, 4) */
    for (i = 0; i < 3; ++i) {
        t = y * y;
        t = t * y;
        t = M * t;
        t = 1.0 - t;
        t = t * y;
        t = t * third;
        y = y + t;
    }
    c = M * y;
    c = c * y;
    r = c * c;
    r = r * c;
    r = r - M;
    t = y * y;
    t = t * third;
    t = r * t;
    c = c - t;
    /* c * 2^q, exact (q within the normal exponent range here) */
    return c * bitsd((uint64_t)(1023 + q) << 52);
}

/* Radius of a sphere of volume v: r = cbrt(v * 3/(4 pi)). */
#define SDMO_THREE_OVER_FOUR_PI 0.238732414637843003
double sdmo_radius(double v)
{
    double t = v * SDMO_THREE_OVER_FOUR_PI;
    return sdmo_cbrt(t);
}

/* Terminal velocity (project definition): three power-law regimes
 * k1 r^2 (Stokes), k2 r, k3 sqrt(r) with the textbook coefficients
 * k1 = 1.19e8 1/(m s), k2 = 8e3 1/s, k3 = 201 m^0.5/s; the regime borders are
 * placed where neighbouring laws meet (r12 = k2/k1, r23 = (k3/k2)^2), so vt is
 * continuous. */
#define SDMO_K1 1.19e8
#define SDMO_K2 8.0e3
#define SDMO_K3 201.0
/* the regime borders written out: r12 = k2/k1 and r23 = (k3/k2)^2 as rounded
 * in double (k2/k1 rounded, then k3/k2 rounded and squared) */
#define SDMO_R12 6.722689075630252e-05
#define SDMO_R23 0.0006312656250000001
double sdmo_terminal_velocity(double r)
{
    double r12 = SDMO_R12;
    double r23 = SDMO_R23;
    if (r < r12) {
        double a = SDMO_K1 * r;
        return a * r;
    }
    if (r < r23) return SDMO_K2 * r;
    return SDMO_K3 * sqrt(r);
}

/* Collision efficiency E(R, q), R = larger radius, q = smaller/larger in
 * (0, 1].  Project table: 12 collector radii x 11 uniform q nodes, values
 * (3 decimals) of the smooth form R^2/(R^2 + (25 um)^2) * (1 - (1-q)^2);
 * bilinear interpolation, clamped to the first/last radius node. */
#define SDMO_NR 12
#define SDMO_NQ 11
static const double sdmo_eff_R[SDMO_NR] = {
    10e-6, 20e-6, 30e-6, 40e-6, 50e-6, 60e-6, 80e-6, 100e-6, 150e-6, 200e-6, 300e-6, 1000e-6};
static const double sdmo_eff_E[SDMO_NR][SDMO_NQ] = {
    {0.000, 0.026, 0.050, 0.070, 0.088, 0.103, 0.116, 0.126, 0.132, 0.137, 0.138},
    {0.000, 0.074, 0.140, 0.199, 0.250, 0.293, 0.328, 0.355, 0.375, 0.386, 0.390},
    {0.000, 0.112, 0.212, 0.301, 0.378, 0.443, 0.496, 0.537, 0.567, 0.584, 0.590},
    {0.000, 0.137, 0.259, 0.367, 0.460, 0.539, 0.604, 0.654, 0.690, 0.712, 0.719},
    {0.000, 0.152, 0.288, 0.408, 0.512, 0.600, 0.672, 0.728, 0.768, 0.792, 0.800},
    {0.000, 0.162, 0.307, 0.435, 0.545, 0.639, 0.716, 0.775, 0.818, 0.844, 0.852},
    {0.000, 0.173, 0.328, 0.465, 0.583, 0.683, 0.765, 0.829, 0.875, 0.902, 0.911},
    {0.000, 0.179, 0.339, 0.480, 0.602, 0.706, 0.791, 0.856, 0.904, 0.932, 0.941},
    {0.000, 0.185, 0.350, 0.496, 0.623, 0.730, 0.817, 0.885, 0.934, 0.963, 0.973},
    {0.000, 0.187, 0.354, 0.502, 0.630, 0.738, 0.827, 0.896, 0.945, 0.975, 0.985},
    {0.000, 0.189, 0.358, 0.506, 0.636, 0.745, 0.834, 0.904, 0.953, 0.983, 0.993},
    {0.000, 0.190, 0.360, 0.510, 0.640, 0.750, 0.839, 0.909, 0.959, 0.989, 0.999},
};

double sdmo_efficiency(double R, double q)
{
    int i, j;
    double t, s, w, e0, e1;
    if (R <= sdmo_eff_R[0]) {
        i = 0; t = 0.0;
    } else if (R >= sdmo_eff_R[SDMO_NR - 1]) {
        i = SDMO_NR - 2; t = 1.0;
    } else {
        i = 0;
        while (sdmo_eff_R[i + 1] <= R) ++i;
        {
            double num = R - sdmo_eff_R[i];
            double den = sdmo_eff_R[i + 1] - sdmo_eff_R[i];
            t = num / den;
        }
    }
    s = q * 10.0;
    j = (int)floor(s);
    if (j >= SDMO_NQ - 1) { j = SDMO_NQ - 2; w = 1.0; }
    else w = s - (double)j;
    {
        double d0 = sdmo_eff_E[i][j + 1] - sdmo_eff_E[i][j];
        double d1 = sdmo_eff_E[i + 1][j + 1] - sdmo_eff_E[i + 1][j];
        double a0 = w * d0, a1 = w * d1;
        double de;
        e0 = sdmo_eff_E[i][j] + a0;
        e1 = sdmo_eff_E[i + 1][j] + a1;
        de = e1 - e0;
        de = t * de;
        return e0 + de;
    }
}

/* Collision efficiency under an electric field (project definition).  Sec. 4 compares
 * with a case of Berry (1966) run with a parametric kernel for electric-field effects on
 * the collision probability, and gives no formula; here the field raises the efficiency
 * toward one: E_eps = E + eps (1 - E), field parameter eps in [0, 1] (eps = 0: E itself;
 * eps = 1: every geometric encounter coalesces). */
double sdmo_efficiency_field(double R, double q, double eps)
{
    double E = sdmo_efficiency(R, q);
    double g = 1.0 - E;
    g = eps * g;
    return E + g;
}

#define SDMO_PI 3.14159265358979311600
/* Hydrodynamic kernel pi (r1 + r2)^2 |vt1 - vt2| E, with E the table efficiency
 * (field = 0) or the field-raised one (field = 1, parameter eps). */
static double hydro_kernel(double v1, double v2, int field, double eps)
{
    double r1 = sdmo_radius(v1), r2 = sdmo_radius(v2);
    double vt1 = sdmo_terminal_velocity(r1), vt2 = sdmo_terminal_velocity(r2);
    double R = r1 > r2 ? r1 : r2;
    double rs = r1 > r2 ? r2 : r1;
    double q = rs / R;
    double E = field ? sdmo_efficiency_field(R, q, eps) : sdmo_efficiency(R, q);
    double s = r1 + r2;
    double a = s * s;
    double dv = vt1 - vt2;
    double K;
    a = SDMO_PI * a;
    dv = fabs(dv);
    K = a * dv;
    return K * E;
}

/* Gravitational (hydrodynamic) kernel: pi (r1 + r2)^2 |vt1 - vt2| E. */
double sdmo_kernel_gravitational(double v1, double v2)
{
    return hydro_kernel(v1, v2, 0, 0.0);
}

/* Electric-field kernel: the gravitational kernel with the efficiency E_eps. */
double sdmo_kernel_electric(double v1, double v2, double eps)
{
    return hydro_kernel(v1, v2, 1, eps);
}

double sdmo_kernel(int kid, double v1, double v2, double golovin_b, double efield)
{
    if (kid == KERNEL_GOLOVIN) return sdmo_kernel_golovin(v1, v2, golovin_b);
    if (kid == KERNEL_ELECTRIC) return sdmo_kernel_electric(v1, v2, efield);
    return sdmo_kernel_gravitational(v1, v2);
}

/* ------------------------------------------------------------------------ */
/* Eq. (p) pieces and Step 3 decision.                                       */
/* ------------------------------------------------------------------------ */

/* Ratio of all non-overlapping pairs (n^2 - n)/2 to candidate pairs
 * floor(n/2), eq. (p). */
double sdmo_pair_scale(uint64_t n)
{
    uint64_t all_pairs = n * (n - 1) / 2;
    uint64_t cand = n / 2;
    return (double)all_pairs / (double)cand;
}

/* p = a(v_j, v_k) max(xi_j, xi_k) * scale * (dt / dV), eq. (p), evaluated as
 * the workflow does: coalescence_kernel, then times_max, then normalize. */
double sdmo_pair_prob(double K, uint64_t xi_a, uint64_t xi_b, double scale, double dt, double dv)
{
    uint64_t xmax = xi_a > xi_b ? xi_a : xi_b;
    double p = K;
    double dtdv = dt / dv;
    p = p * (double)xmax;   /* times_max */
    p = p * scale;          /* normalize: pair-count ratio ... */
    p = p * dtdv;           /* ... and dt / dV */
    return p;
}

/* gamma~ = min(ceil(p - phi), floor(xi_j / xi_k)) with xi_j >= xi_k
 * (eq. gamma2).  ceil(p - phi) is evaluated as floor(p) + [phi < p - floor(p)],
 * which is the same integer for phi in [0,1) and needs no rounded subtraction
 * p - phi.  When floor(p) already reaches the cap the cap is returned without
 * converting p to an integer. */
uint64_t sdmo_gamma_tilde(double p, double phi, uint64_t xi_j, uint64_t xi_k)
{
    uint64_t cap = xi_j / xi_k;
    double fl = floor(p);
    double frac = p - fl;
    uint64_t g;
    if (fl >= (double)cap) return cap;
    g = (uint64_t)fl + (phi < frac ? 1u : 0u);
    return g < cap ? g : cap;
}

/* Attribute update of one pair, eqs. (coal_attr_0)/(coal) with the update
 * routine's conventions: j is the first SD of the pair unless its
 * multiplicity is smaller than the second's; g == 0 leaves both untouched.
 * attr is [n_attr][stride].  Returns gamma~ (0 = no collision). */
uint64_t sdmo_update_pair(uint64_t* xi, double* attr, uint32_t n_attr, uint64_t stride,
                          uint64_t first, uint64_t second, double p, double phi)
{
    uint64_t j = first, k = second, g, new_n;
    uint32_t a;
    if (xi[j] < xi[k]) { uint64_t t = j; j = k; k = t; }
    g = sdmo_gamma_tilde(p, phi, xi[j], xi[k]);
    if (g == 0) return 0;
    new_n = xi[j] - g * xi[k];
    if (new_n > 0) {                                  /* case 1 */
        xi[j] = new_n;
        for (a = 0; a < n_attr; ++a) {
            double t = (double)g * attr[a * stride + j];
            attr[a * stride + k] = t + attr[a * stride + k];
        }
    } else {                                          /* case 2 */
        xi[j] = xi[k] / 2;
        xi[k] = xi[k] - xi[j];
        for (a = 0; a < n_attr; ++a) {
            double t = (double)g * attr[a * stride + j];
            attr[a * stride + j] = t + attr[a * stride + k];
            attr[a * stride + k] = attr[a * stride + j];
        }
    }
    return g;
}

/* ------------------------------------------------------------------------ */
/* One full timestep, Fig. "fig:algo".                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t n_pairs;        /* candidate pairs examined */
    uint64_t n_collisions;   /* pairs with gamma~ > 0 */
    uint64_t n_removed;      /* SDs whose multiplicity became 0 */
    uint64_t sum_gamma;      /* sum of gamma~ */
} sdmo_stats;

typedef struct { uint32_t key; uint32_t pos; uint32_t slot; } key_rec;

static int cmp_key_rec(const void* a, const void* b)
{
    const key_rec* x = (const key_rec*)a;
    const key_rec* y = (const key_rec*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

#define SDMO_SHUFFLE_SORT 0
#define SDMO_SHUFFLE_PRP 1

/* Stable compaction of every cell: live SDs to the front in slot order, freed
 * slots get xi = 0 and attributes 0. */
void sdmo_compact(uint64_t n_slots, uint32_t n_cell, const uint32_t* cell_start, uint64_t* xi, double* attr,
                  uint32_t n_attr)
{
    uint32_t c, a;
    for (c = 0; c < n_cell; ++c) {
        uint64_t dst = cell_start[c], src;
        for (src = cell_start[c]; src < cell_start[c + 1]; ++src) {
            if (xi[src] == 0) continue;
            if (dst != src) {
                xi[dst] = xi[src];
                for (a = 0; a < n_attr; ++a) attr[a * n_slots + dst] = attr[a * n_slots + src];
            }
            ++dst;
        }
        for (; dst < cell_start[c + 1]; ++dst) {
            xi[dst] = 0;
            for (a = 0; a < n_attr; ++a) attr[a * n_slots + dst] = 0.0;
        }
    }
}

/*
 * xi[n_slots], attr[n_attr][n_slots] (attr 0 = volume), cell_start[n_cell+1],
 * dv[n_cell], kernel_id[n_cell].  In-place update of xi and attr.
 */
int sdmo_step(uint64_t n_slots, uint32_t n_cell, const uint32_t* cell_start,
              uint64_t* xi, double* attr, uint32_t n_attr,
              const double* dv, const uint8_t* kernel_id, double golovin_b, double efield,
              double dt, uint64_t seed, uint32_t step, int shuffle, sdmo_stats* stats)
{
    uint32_t c;
    sdmo_stats st = {0, 0, 0, 0};
    uint64_t max_cell = 0;
    key_rec* list;
    uint64_t* order;
    double* pair_prob;
    for (c = 0; c < n_cell; ++c) {
        uint64_t w = cell_start[c + 1] - cell_start[c];
        if (cell_start[c + 1] < cell_start[c]) return SDMO_EINVAL;
        if (w > max_cell) max_cell = w;
    }
    if (cell_start[n_cell] > n_slots) return SDMO_EINVAL;
    if (shuffle != SDMO_SHUFFLE_SORT && shuffle != SDMO_SHUFFLE_PRP) return SDMO_EINVAL;
    list = (key_rec*)malloc((max_cell + 1) * sizeof(key_rec));
    order = (uint64_t*)malloc((max_cell + 1) * sizeof(uint64_t));
    pair_prob = (double*)malloc((max_cell / 2 + 1) * sizeof(double));
    if (!list || !order || !pair_prob) { free(list); free(order); free(pair_prob); return SDMO_ENOMEM; }

    for (c = 0; c < n_cell; ++c) {
        uint64_t base = cell_start[c];
        uint32_t width = cell_start[c + 1] - cell_start[c];
        uint32_t n = 0, l, m, q, npairs;
        double scale;
        /* step 0: remove_if_equal_0 -- the cell's list L_c holds live SDs only */
        for (l = 0; l < width; ++l)
            if (xi[base + l] != 0) { list[n].pos = n; list[n].slot = l; ++n; }
        if (n < 2) continue;
        /* step 1: urand + shuffle_per_cell: the shuffled list as slot offsets */
        if (shuffle == SDMO_SHUFFLE_SORT || n < SDMO_PRP_MIN_N) {
            for (q = 0; q < n; ++q) list[q].key = sdmo_shuffle_key(seed, c, step, list[q].pos);
            qsort(list, n, sizeof(key_rec), cmp_key_rec);
            for (q = 0; q < n; ++q) order[q] = base + list[q].slot;
        } else {
            uint32_t K[SDMO_PRP_ROUNDS];
            sdmo_prp_keys(seed, c, step, K);
            for (q = 0; q < n; ++q) order[q] = base + list[sdmo_prp(q, n, K)].slot;
        }
        /* flag_pairs: pair m = (L'[2m], L'[2m+1]) */
        npairs = n / 2;
        /* step 2: coalescence_kernel, times_max, normalize */
        for (m = 0; m < npairs; ++m) {
            double v1 = attr[order[2 * m]];
            double v2 = attr[order[2 * m + 1]];
            pair_prob[m] = sdmo_kernel(kernel_id ? kernel_id[c] : KERNEL_GOLOVIN, v1, v2, golovin_b, efield);
        }
        scale = sdmo_pair_scale(n);
        for (m = 0; m < npairs; ++m) {
            uint64_t a = xi[order[2 * m]], b = xi[order[2 * m + 1]];
            pair_prob[m] = sdmo_pair_prob(pair_prob[m], a, b, scale, dt, dv[c]);
        }
        /* step 3: urand, compute_gamma, update_attributes */
        for (m = 0; m < npairs; ++m) {
            double phi = sdmo_phi(seed, c, step, m);
            uint64_t j = order[2 * m], k = order[2 * m + 1];
            uint64_t g = sdmo_update_pair(xi, attr, n_attr, n_slots, j, k, pair_prob[m], phi);
            st.n_pairs++;
            if (g) {
                st.n_collisions++;
                st.sum_gamma += g;
                if (xi[j] == 0) st.n_removed++;
                if (xi[k] == 0) st.n_removed++;
            }
        }
    }
    free(list);
    free(order);
    free(pair_prob);
    /* the removals take effect in the storage (Step 0 of the next step) */
    sdmo_compact(n_slots, n_cell, cell_start, xi, attr, n_attr);
    if (stats) *stats = st;
    return SDMO_OK;
}

/* Many steps: step indices step0 .. step0 + n_steps - 1. */
int sdmo_run(uint64_t n_slots, uint32_t n_cell, const uint32_t* cell_start,
             uint64_t* xi, double* attr, uint32_t n_attr,
             const double* dv, const uint8_t* kernel_id, double golovin_b, double efield,
             double dt, uint64_t seed, uint32_t step0, uint32_t n_steps, int shuffle, sdmo_stats* total)
{
    uint32_t s;
    sdmo_stats acc = {0, 0, 0, 0}, st;
    for (s = 0; s < n_steps; ++s) {
        int rc = sdmo_step(n_slots, n_cell, cell_start, xi, attr, n_attr, dv, kernel_id,
                           golovin_b, efield, dt, seed, step0 + s, shuffle, &st);
        if (rc) return rc;
        acc.n_pairs += st.n_pairs;
        acc.n_collisions += st.n_collisions;
        acc.n_removed += st.n_removed;
        acc.sum_gamma += st.sum_gamma;
    }
    if (total) *total = acc;
    return SDMO_OK;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics.                                                              */
/* ------------------------------------------------------------------------ */

/* Totals over live SDs: sums[0] = sum xi (exact, returned via n_total),
 * sums[1] = sum xi * v (compensated summation), n_live. */
void sdmo_totals(uint64_t n_slots, const uint64_t* xi, const double* v,
                 uint64_t* n_total, uint64_t* n_live, double* mass)
{
    uint64_t i, tot = 0, live = 0;
    double s = 0.0, comp = 0.0;
    for (i = 0; i < n_slots; ++i) {
        if (xi[i] == 0) continue;
        {
            double t = (double)xi[i] * v[i];
            double y = t - comp;
            double z = s + y;
            comp = (z - s) - y;
            s = z;
        }
        tot += xi[i];
        ++live;
    }
    *n_total = tot;
    *n_live = live;
    *mass = s;
}

/* ------------------------------------------------------------------------ */
/* Golovin analytic solution (Sec. 4).                                       */
/* ------------------------------------------------------------------------ */

/* Exponentially scaled modified Bessel function of the first kind, order 1:
 * I1e(x) = exp(-|x|) I1(x), x >= 0.  Power series sum_k (x/2)^(2k+1) /
 * (k! (k+1)!) below x = 30; Hankel large-argument expansion (A&S 9.7.1,
 * mu = 4) above. */
double sdmo_i1e(double x)
{
    if (x < 0) return -sdmo_i1e(-x);
    if (x < 30.0) {
        double h = 0.5 * x, term = h, sum = h;
        int k;
        for (k = 1; k < 200; ++k) {
            term = term * h * h / ((double)k * (double)(k + 1));
            sum += term;
            if (term < sum * 1e-17) break;
        }
        return sum * exp(-x);
    } else {
        /* 1/sqrt(2 pi x) * sum_k (-1)^k prod_{i=1..k} (mu - (2i-1)^2) / (k! (8x)^k) */
        double mu = 4.0, z8 = 8.0 * x, term = 1.0, sum = 1.0;
        int k;
        for (k = 1; k < 30; ++k) {
            double odd = (double)(2 * k - 1);
            double nt = -term * (mu - odd * odd) / ((double)k * z8);
            if (fabs(nt) > fabs(term)) break;   /* asymptotic series: stop at smallest term */
            term = nt;
            sum += term;
            if (fabs(term) < 1e-17 * fabs(sum)) break;
        }
        return sum / sqrt(2.0 * 3.14159265358979323846 * x);
    }
}

/* Number density per unit volume-of-particle, normalised to 1 at t = 0:
 * phi(v,t) = (1 - tau) / (v sqrt(tau)) I1e(2 v sqrt(tau)/vbar)
 *            exp(-v (1 + tau - 2 sqrt(tau)) / vbar),
 * tau = 1 - exp(-N0 b vbar t).  At t = 0 it is exp(-v/vbar)/vbar. */
double sdmo_golovin_phi(double v, double t, double vbar, double n0, double b)
{
    double tau = 1.0 - exp(-n0 * b * vbar * t);
    double st;
    if (t <= 0.0) return exp(-v / vbar) / vbar;
    st = sqrt(tau);
    return (1.0 - tau) / (v * st) * sdmo_i1e(2.0 * v * st / vbar)
           * exp(-v * (1.0 + tau - 2.0 * st) / vbar);
}
