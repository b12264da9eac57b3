// sdm_math.cuh -- device arithmetic of the SDM coalescence step (sm_103a).
//
// Three layers:
//  * Philox4x32-10 (Salmon et al., SC'11) for the shuffle keys and phi.
//  * The FP64 path: collision kernels and eq. (p) written with explicit
//    round-to-nearest intrinsics (__dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn)
//    so that no operation is contracted or reordered; its results are the
//    documented operation order evaluated in IEEE double.  B300 executes FP64
//    at a small fraction of its FP32 rate, so this path only runs for pairs
//    the FP32 path below cannot settle.
//  * The FP32 path: the same quantities in single precision together with a
//    bound err such that |p64 - p32| <= err.  The integer outcome gamma of
//    Step 3 is taken from [p32 - err, p32 + err] whenever that interval
//    settles it (the usual case), which gives exactly the FP64 result.
#pragma once
#include <cstdint>

namespace sdm {

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// The key schedule of Philox4x32-10 for one key: round r uses (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85) mod 2^32.  Worked out once on the host and passed with a launch's
// arguments, so that every round reads its two key words as operands instead of adding them.
struct PhiloxKeys { uint32_t k0[10], k1[10]; };

inline PhiloxKeys philox_keys_host(uint32_t k0, uint32_t k1)
{
    PhiloxKeys K{};
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        K.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}

// philox() with the schedule of the key given beforehand (the same result)
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const PhiloxKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ K.k0[r];
        const uint32_t n2 = hi0 ^ c3 ^ K.k1[r];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t u4_word(const U4& x, uint32_t i)
{
    return i == 0 ? x.x : i == 1 ? x.y : i == 2 ? x.z : x.w;
}

// 53-bit integer of phi for candidate pair m (phi = u53 * 2^-53).
__device__ __forceinline__ uint64_t phi_u53(const PhiloxKeys& K, uint32_t cell, uint32_t step, uint32_t m)
{
    const U4 x = philox(m >> 1, cell, step, 1u, K);
    const uint32_t hi = (m & 1u) ? x.z : x.x;
    const uint32_t lo = (m & 1u) ? x.w : x.y;
    return ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
}

// ---------------------------------------------------------------------------
// PRP shuffle: a keyed bijection P of [0, n) for cells of more than 256 live
// SDs -- an eight-round alternating Feistel network on Z_A x Z_B with round
// function h = lowbias32(v ^ K_r) without its last xor-shift (C. Wellons'
// 32-bit integer hash) of the other half v, added as floor(h M / 2^32) modulo
// the half's size M.  For
// n = 2^k the halves have floor(k/2) and k - floor(k/2) bits (A B = n);
// otherwise A = ceil(sqrt n), B = ceil(n / A).  Philox round keys;
// cycle-walking into [0, n), rare because A B < n + A.
// The shuffled list is L'[q] = L[P(q)]: the SDs of pair m are found directly,
// with no sort and no data movement.
// ---------------------------------------------------------------------------
constexpr uint32_t PRP_ROUNDS = 8;
constexpr uint32_t PRP_MIN_N = 257;      // smaller cells are shuffled by sorting keys

// The round function h(v ^ K) of the bijection: lowbias32 (C. Wellons' 32-bit
// integer hash) without its last step x ^= x >> 16 -- a round uses floor(h M /
// 2^32), M < 2^16, which the top bits of h decide (alone when M is a power of
// two), and that step leaves the top 16 bits unchanged.  The halves have at most
// 16 bits, so (v ^ K) >> 16 = K >> 16 and the hash's first step x ^= x >> 16 is
// folded into the round key: h = lowbias32_top16(v ^ Kx), Kx = K ^ (K >> 16).
__device__ __forceinline__ uint32_t lowbias32_top16(uint32_t x)
{
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    return x;
}

struct Prp {
    uint32_t K[PRP_ROUNDS];       // folded round keys Kx = K ^ (K >> 16)
    uint32_t n;                   // list length (walk bound)
    uint32_t A, B, Binv;          // domain Z_A x Z_B, Binv = ceil(2^32 / B)
    uint32_t pow2;                // A = 2^a and B = 2^b: the same rounds by shifts and masks
    uint32_t b, sa, sb;           //   x = L 2^b + R; floor(h A / 2^32) = h >> sa, h B likewise
};

__device__ __forceinline__ uint32_t prp_bits(uint32_t n)
{
    return n <= 1 ? 0u : 32u - (uint32_t)__clz(n - 1u);   // ceil(log2 n)
}

// Domain of the network for a list of n elements (x = L B + R, L < A, R < B):
// n = 2^k: A = 2^floor(k/2), B = 2^(k - floor(k/2)); otherwise A = ceil(sqrt n),
// B = ceil(n / A), so that n <= A B < n + A and cycle-walking is rare.
__device__ __forceinline__ void prp_domain_of(uint32_t n, uint32_t& A, uint32_t& B)
{
    if (n != 0 && (n & (n - 1)) == 0) {
        const uint32_t k = prp_bits(n), a = k >> 1;
        A = 1u << a;
        B = 1u << (k - a);
    } else {
        uint32_t r = (uint32_t)ceilf(sqrtf((float)n));
        while ((uint64_t)r * r < n) ++r;
        while (r > 1 && (uint64_t)(r - 1) * (r - 1) >= n) --r;
        A = r;
        B = (n + r - 1) / r;
    }
}

__device__ __forceinline__ void prp_set_domain(Prp& P, uint32_t n)
{
    P.n = n;
    prp_domain_of(n, P.A, P.B);
    P.Binv = P.B > 1 ? (uint32_t)((0x100000000ull + P.B - 1) / P.B) : 0u;   // B = 1 only for n = 1
    P.pow2 = (n != 0 && (n & (n - 1)) == 0) ? 1u : 0u;
    const uint32_t a = 31u - __clz(P.A);
    P.b = 31u - __clz(P.B);
    P.sa = a ? 32u - a : 31u;     // A = 1: the mask A - 1 = 0 clears the shifted hash
    P.sb = P.b ? 32u - P.b : 31u;
}

// whether the network for n elements is the one P holds (only the walk bound differs)
__device__ __forceinline__ bool prp_same_network(const Prp& P, uint32_t n)
{
    uint32_t A, B;
    prp_domain_of(n, A, B);
    return A == P.A && B == P.B;
}

// x / B and x mod B for x < A B
__device__ __forceinline__ void prp_split(const Prp& P, uint32_t x, uint32_t& L, uint32_t& R)
{
    uint32_t q = __umulhi(x, P.Binv);            // floor(x / B) or one more
    if (q * P.B > x) --q;
    L = q;
    R = x - q * P.B;
}

// one round pair of the network: L = (L + floor(h A / 2^32)) mod A, then R likewise mod B
__device__ __forceinline__ void prp_round_pair(const Prp& P, uint32_t kl, uint32_t kr, uint32_t& L, uint32_t& R)
{
    const uint32_t tl = L + __umulhi(lowbias32_top16(R ^ kl), P.A);
    L = tl >= P.A ? tl - P.A : tl;
    const uint32_t tr = R + __umulhi(lowbias32_top16(L ^ kr), P.B);
    R = tr >= P.B ? tr - P.B : tr;
}

// The same round pair when A = 2^a and B = 2^b (a, b <= 16): floor(h A / 2^32) is
// the top a bits of h, and the reduction mod A is deferred -- L and R carry values
// congruent to the halves (below 2^19 after the four additions of a pass) and are
// masked where read.
__device__ __forceinline__ void prp_round_pair_pow2(const Prp& P, uint32_t kl, uint32_t kr, uint32_t& L, uint32_t& R)
{
    L += lowbias32_top16((R & (P.B - 1u)) ^ kl) >> P.sa;
    R += lowbias32_top16((L & (P.A - 1u)) ^ kr) >> P.sb;
}

__device__ __forceinline__ void prp_init(Prp& P, const PhiloxKeys& Kp, uint32_t cell, uint32_t step, uint32_t n)
{
    const U4 x = philox(0u, cell, step, 2u, Kp);
    const U4 y = philox(1u, cell, step, 2u, Kp);
    const uint32_t K[PRP_ROUNDS] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
#pragma unroll
    for (int r = 0; r < (int)PRP_ROUNDS; ++r) P.K[r] = K[r] ^ (K[r] >> 16);
    prp_set_domain(P, n);
}

__device__ __forceinline__ uint32_t feistel(const Prp& P, uint32_t q)
{
    uint32_t L, R;
    prp_split(P, q, L, R);
#pragma unroll
    for (uint32_t r = 0; r < PRP_ROUNDS; r += 2) prp_round_pair(P, P.K[r], P.K[r + 1], L, R);
    return L * P.B + R;
}

// P(q) for q < n (cycle-walking terminates: q's cycle contains q itself)
__device__ __forceinline__ uint32_t prp_map(const Prp& P, uint32_t q)
{
    uint32_t e = feistel(P, q);
    while (e >= P.n) e = feistel(P, e);
    return e;
}

// ---------------------------------------------------------------------------
// Constants of the kernels (each written out here from the definitions).
// ---------------------------------------------------------------------------
constexpr double THREE_OVER_FOUR_PI = 0.238732414637843003;
constexpr double PI_D = 3.14159265358979311600;
constexpr double VT_K1 = 1.19e8;   // Stokes regime, 1/(m s)
constexpr double VT_K2 = 8.0e3;    // linear regime, 1/s
constexpr double VT_K3 = 201.0;    // square-root regime, m^0.5/s
constexpr int EFF_NR = 12;
constexpr int EFF_NQ = 11;

// collector radius nodes [m] and efficiency values E[R][q], q = 0, 0.1, ..., 1
#define SDM_EFF_RADII(X) X(10e-6) X(20e-6) X(30e-6) X(40e-6) X(50e-6) X(60e-6) X(80e-6) X(100e-6) X(150e-6) \
    X(200e-6) X(300e-6) X(1000e-6)
#define SDM_EFF_VALUES(X) \
    X(0.000) X(0.026) X(0.050) X(0.070) X(0.088) X(0.103) X(0.116) X(0.126) X(0.132) X(0.137) X(0.138) \
    X(0.000) X(0.074) X(0.140) X(0.199) X(0.250) X(0.293) X(0.328) X(0.355) X(0.375) X(0.386) X(0.390) \
    X(0.000) X(0.112) X(0.212) X(0.301) X(0.378) X(0.443) X(0.496) X(0.537) X(0.567) X(0.584) X(0.590) \
    X(0.000) X(0.137) X(0.259) X(0.367) X(0.460) X(0.539) X(0.604) X(0.654) X(0.690) X(0.712) X(0.719) \
    X(0.000) X(0.152) X(0.288) X(0.408) X(0.512) X(0.600) X(0.672) X(0.728) X(0.768) X(0.792) X(0.800) \
    X(0.000) X(0.162) X(0.307) X(0.435) X(0.545) X(0.639) X(0.716) X(0.775) X(0.818) X(0.844) X(0.852) \
    X(0.000) X(0.173) X(0.328) X(0.465) X(0.583) X(0.683) X(0.765) X(0.829) X(0.875) X(0.902) X(0.911) \
    X(0.000) X(0.179) X(0.339) X(0.480) X(0.602) X(0.706) X(0.791) X(0.856) X(0.904) X(0.932) X(0.941) \
    X(0.000) X(0.185) X(0.350) X(0.496) X(0.623) X(0.730) X(0.817) X(0.885) X(0.934) X(0.963) X(0.973) \
    X(0.000) X(0.187) X(0.354) X(0.502) X(0.630) X(0.738) X(0.827) X(0.896) X(0.945) X(0.975) X(0.985) \
    X(0.000) X(0.189) X(0.358) X(0.506) X(0.636) X(0.745) X(0.834) X(0.904) X(0.953) X(0.983) X(0.993) \
    X(0.000) X(0.190) X(0.360) X(0.510) X(0.640) X(0.750) X(0.839) X(0.909) X(0.959) X(0.989) X(0.999)
#define SDM_AS_DOUBLE(v) v,
#define SDM_AS_FLOAT(v) (float)(v),
__constant__ double c_eff_R[EFF_NR] = {SDM_EFF_RADII(SDM_AS_DOUBLE)};
__constant__ double c_eff_E[EFF_NR * EFF_NQ] = {SDM_EFF_VALUES(SDM_AS_DOUBLE)};
// the same table rounded to float (the FP32 path stages it in shared memory)
__constant__ float c_eff_Rf[EFF_NR] = {SDM_EFF_RADII(SDM_AS_FLOAT)};
__constant__ float c_eff_Ef[EFF_NR * EFF_NQ] = {SDM_EFF_VALUES(SDM_AS_FLOAT)};
// 1 / (R[i+1] - R[i]) rounded to float (last entry unused)
#define SDM_INV_DR(i) (float)(1.0 / (c_eff_R_h[(i) + 1] - c_eff_R_h[i]))
constexpr double c_eff_R_h[EFF_NR] = {SDM_EFF_RADII(SDM_AS_DOUBLE)};
__constant__ float c_eff_invdRf[EFF_NR] = {SDM_INV_DR(0), SDM_INV_DR(1), SDM_INV_DR(2), SDM_INV_DR(3), SDM_INV_DR(4),
                                           SDM_INV_DR(5), SDM_INV_DR(6), SDM_INV_DR(7), SDM_INV_DR(8), SDM_INV_DR(9),
                                           SDM_INV_DR(10), 0.f};


// ---------------------------------------------------------------------------
// FP64 path (documented operation order, no contraction)
// ---------------------------------------------------------------------------

// Cube root from + and * only: x = m 2^e, m in [0.5, 1), e = 3q + rmd; seed
// y = ((0.456419 m - 1.19161) m + 1.73758) 2^(-rmd/3) ~ m^(-1/3); M = m 2^rmd;
// three Newton steps y <- y + y (1 - M y^3)/3; c = (M y) y; one residual
// correction c <- c - (c^3 - M) y^2/3; result c 2^q.  Positive normal x.
__device__ __forceinline__ double cbrt_d(double x)
{
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ff) - 1022;
    const double m = __longlong_as_double((long long)((u & 0x800fffffffffffffull) | (1022ull << 52)));
    const int q = (e >= 0) ? e / 3 : -((-e + 2) / 3);
    const int rmd = e - 3 * q;
    const double third = 0.3333333333333333;
    double y = __dmul_rn(0.456419, m);
    y = __dsub_rn(y, 1.19161);
    y = __dmul_rn(y, m);
    y = __dadd_rn(y, 1.73758);
    y = __dmul_rn(y, rmd == 0 ? 1.0 : (rmd == 1 ? 0.7937005259840998 : 0.6299605249474366));
    const double M = rmd == 1 ? __dmul_rn(m, 2.0) : (rmd == 2 ? __dmul_rn(m, 4.0) : m);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double t = __dmul_rn(y, y);
        t = __dmul_rn(t, y);
        t = __dmul_rn(M, t);
        t = __dsub_rn(1.0, t);
        t = __dmul_rn(t, y);
        t = __dmul_rn(t, third);
        y = __dadd_rn(y, t);
    }
    double c = __dmul_rn(M, y);
    c = __dmul_rn(c, y);
    double r = __dmul_rn(c, c);
    r = __dmul_rn(r, c);
    r = __dsub_rn(r, M);
    double t = __dmul_rn(y, y);
    t = __dmul_rn(t, third);
    t = __dmul_rn(r, t);
    c = __dsub_rn(c, t);
    return __dmul_rn(c, __longlong_as_double((long long)((uint64_t)(1023 + q) << 52)));
}

__device__ __forceinline__ double radius_d(double v)
{
    return cbrt_d(__dmul_rn(v, THREE_OVER_FOUR_PI));
}

// regime borders k2/k1 and (k3/k2)^2 as rounded in double, written out
constexpr double VT_R12 = 6.722689075630252e-05;
constexpr double VT_R23 = 0.0006312656250000001;

__device__ __forceinline__ double vt_d(double r)
{
    const double r12 = VT_R12;
    const double r23 = VT_R23;
    if (r < r12) return __dmul_rn(__dmul_rn(VT_K1, r), r);
    if (r < r23) return __dmul_rn(VT_K2, r);
    return __dmul_rn(VT_K3, __dsqrt_rn(r));
}

// interval index i with R[i] <= R < R[i+1], for R[0] < R < R[EFF_NR-1]: the
// comparisons are independent (FP64 compares have long latency on B300)
__device__ __forceinline__ int eff_interval_d(double R)
{
    int i = 0;
#pragma unroll
    for (int k = 1; k < EFF_NR - 1; ++k) i += (R >= c_eff_R[k]) ? 1 : 0;
    return i;
}

__device__ __forceinline__ double efficiency_d(double R, double q)
{
    int i;
    double t;
    if (R <= c_eff_R[0]) {
        i = 0; t = 0.0;
    } else if (R >= c_eff_R[EFF_NR - 1]) {
        i = EFF_NR - 2; t = 1.0;
    } else {
        i = eff_interval_d(R);
        t = __ddiv_rn(__dsub_rn(R, c_eff_R[i]), __dsub_rn(c_eff_R[i + 1], c_eff_R[i]));
    }
    const double s = __dmul_rn(q, 10.0);
    int j = __double2int_rz(s);                        // floor: s >= 0
    double w;
    if (j >= EFF_NQ - 1) { j = EFF_NQ - 2; w = 1.0; }
    else w = __dsub_rn(s, (double)j);
    const double* E = c_eff_E;
    const double d0 = __dsub_rn(E[i * EFF_NQ + j + 1], E[i * EFF_NQ + j]);
    const double d1 = __dsub_rn(E[(i + 1) * EFF_NQ + j + 1], E[(i + 1) * EFF_NQ + j]);
    const double e0 = __dadd_rn(E[i * EFF_NQ + j], __dmul_rn(w, d0));
    const double e1 = __dadd_rn(E[(i + 1) * EFF_NQ + j], __dmul_rn(w, d1));
    return __dadd_rn(e0, __dmul_rn(t, __dsub_rn(e1, e0)));
}

// Hydrodynamic kernel pi (r1+r2)^2 |vt1 - vt2| E: the gravitational kernel (field = false), or the
// electric-field kernel (project definition; Sec. 4 names a parametric kernel for electric-field
// effects without a formula), whose efficiency the field parameter eps in [0, 1] raises toward
// one: E_eps = E + eps (1 - E).
__device__ __noinline__ double kernel_hydro_d(double v1, double v2, bool field, double eps)
{
    const double r1 = radius_d(v1), r2 = radius_d(v2);
    const double vt1 = vt_d(r1), vt2 = vt_d(r2);
    const double R = r1 > r2 ? r1 : r2;
    const double rs = r1 > r2 ? r2 : r1;
    double E = efficiency_d(R, __ddiv_rn(rs, R));
    if (field) E = __dadd_rn(E, __dmul_rn(eps, __dsub_rn(1.0, E)));
    const double s = __dadd_rn(r1, r2);
    double a = __dmul_rn(s, s);
    a = __dmul_rn(PI_D, a);
    const double dv = fabs(__dsub_rn(vt1, vt2));
    return __dmul_rn(__dmul_rn(a, dv), E);
}

__device__ __forceinline__ double kernel_grav_d(double v1, double v2) { return kernel_hydro_d(v1, v2, false, 0.0); }

__device__ __forceinline__ double kernel_golovin_d(double v1, double v2, double b)
{
    return __dmul_rn(b, __dadd_rn(v1, v2));
}

// eq. (p): p = ((a * max(xi)) * scale) * (dt / dV), scale = ((n^2-n)/2) / floor(n/2)
__device__ __forceinline__ double pair_prob_d(double K, uint64_t xmax, uint32_t n, double dt, double dv)
{
    const uint64_t nn = n;
    const uint64_t all_pairs = nn * (nn - 1) / 2;
    const uint64_t cand = nn / 2;
    const double scale = __ddiv_rn(__ull2double_rn(all_pairs), __ull2double_rn(cand));
    const double dtdv = __ddiv_rn(dt, dv);
    double p = K;
    p = __dmul_rn(p, __ull2double_rn(xmax));
    p = __dmul_rn(p, scale);
    p = __dmul_rn(p, dtdv);
    return p;
}

// gamma~ = min(floor(p) + [phi < p - floor(p)], floor(xi_j / xi_k)), Step 3 and eq. (gamma2)
__device__ __forceinline__ uint64_t gamma_tilde_d(double p, uint64_t u53, uint64_t xi_j, uint64_t xi_k)
{
    const uint64_t cap = xi_j / xi_k;
    const double fl = floor(p);
    const double frac = __dsub_rn(p, fl);
    if (fl >= __ull2double_rn(cap)) return cap;
    const double phi = __dmul_rn(__ull2double_rn(u53), 0x1p-53);
    const uint64_t g = (uint64_t)fl + (phi < frac ? 1ull : 0ull);
    return g < cap ? g : cap;
}

__device__ __forceinline__ double kernel_d(uint32_t kid, double v1, double v2, double golovin_b, double efield)
{
    return kid == 0 ? kernel_golovin_d(v1, v2, golovin_b) : kernel_hydro_d(v1, v2, kid == 2, efield);
}

// The whole FP64 decision of one pair: kernel, eq. (p), gamma~.  Kept out of line so
// that none of its (slow on B300) FP64 work is hoisted into the common path.
__device__ __noinline__ uint64_t gamma_tilde_fp64_path(uint32_t kid, double v1, double v2, double golovin_b,
                                                       double efield, uint32_t n, double dt, double dv, uint64_t u53,
                                                       uint64_t xi_j, uint64_t xi_k)
{
    const double K = kernel_d(kid, v1, v2, golovin_b, efield);
    const double p = pair_prob_d(K, xi_j, n, dt, dv);
    return gamma_tilde_d(p, u53, xi_j, xi_k);
}

// ---------------------------------------------------------------------------
// Second filter for the gravitational kernel: p in FP64 from FP32 seeds refined
// by Newton steps -- multiplications and FMAs only, a short dependency chain
// (B300 runs FP64 with long latency, and a division costs several hundred
// cycles) -- with a bound on its distance to the exact sequence's value.  The
// exact sequence above runs only when this interval cannot decide gamma.
//   Error budget relative to B = scale pi (r1+r2)^2 (vt1 + vt2) (u = 2^-53):
//   a radius after one Newton step from cbrtf (seed within 1 ulp of the float
//   cube root of the float-rounded argument: |e0| <= 2^-22.7) with a step
//   factor h = 1/(3 r0^2) from float arithmetic (|eta| <= 2^-21.4): relative
//   error ~ e0^2 + |eta e0| <= 2^-43 ~ 1000u; 1/sqrt(r) after one Newton step
//   from rsqrtf (2 ulp): 1.5 e0^2 ~ 1000u.  (r1+r2)^2, the fall speeds and
//   their difference: ~6000u B; q = rs (1/R) with a refined reciprocal and
//   t = (R - R_i) (1/dR_i), R / dR_i <= 6: weights off by ~12000u, times table
//   steps <= 1 -> ~15000u B; scale with a refined reciprocal of dV: ~10u.  In
//   all below 25000u B ~ 2^-38.4 B; the bound used is 2^-36 B.
// ---------------------------------------------------------------------------
constexpr double LITE_REL_BOUND = 0x1p-36;
// The second filter reads its tables through L1 from global memory: its lookups use
// indices known only at run time, which serialise on the constant cache, and a cold
// constant bank is fetched line by line on the filter's critical path.
__device__ const double g_eff_Rd[EFF_NR] = {SDM_EFF_RADII(SDM_AS_DOUBLE)};
__device__ const double g_eff_Ed[EFF_NR * EFF_NQ] = {SDM_EFF_VALUES(SDM_AS_DOUBLE)};
__device__ const double g_eff_invdRd[EFF_NR] = {
    1.0 / (10e-6), 1.0 / (10e-6), 1.0 / (10e-6), 1.0 / (10e-6), 1.0 / (10e-6), 1.0 / (20e-6),
    1.0 / (20e-6), 1.0 / (50e-6), 1.0 / (50e-6), 1.0 / (100e-6), 1.0 / (700e-6), 0.0};

// 1/d to about 2^-46 relative (d a normal float-range double)
__device__ __forceinline__ double rcp_lite(double d)
{
    const double y0 = (double)__frcp_rn((float)d);
    const double e = __fma_rn(-d, y0, 1.0);
    return __fma_rn(y0, e, y0);
}

__device__ __forceinline__ double cbrt_lite(double x)
{
    const float xf = (float)x;
    const float rf = cbrtf(xf);
    const double r = (double)rf;
    const double h = (double)__frcp_rn(3.0f * __fmul_rn(rf, rf));   // ~ 1 / (3 r^2)
    return __fma_rn(-__fma_rn(r * r, r, -x), h, r);                 // one Newton step
}

__device__ __forceinline__ double vt_lite(double r)
{
    if (r < VT_R12) return VT_K1 * r * r;
    if (r < VT_R23) return VT_K2 * r;
    const double y0 = (double)rsqrtf((float)r);         // 1 / sqrt(r)
    const double y = __fma_rn(0.5 * y0, __fma_rn(-r * y0, y0, 1.0), y0);   // one Newton step
    return VT_K3 * (r * y);
}

__device__ __forceinline__ double efficiency_lite(double R, double q)
{
    int i;
    double t;
    if (R <= c_eff_R[0]) { i = 0; t = 0.0; }                  // fixed indices: constant operands
    else if (R >= c_eff_R[EFF_NR - 1]) { i = EFF_NR - 2; t = 1.0; }
    else {
        i = eff_interval_d(R);
        t = (R - __ldg(&g_eff_Rd[i])) * __ldg(&g_eff_invdRd[i]);
    }
    const double s = q * 10.0;
    int j = __double2int_rz(s);
    double w;
    if (j >= EFF_NQ - 1) { j = EFF_NQ - 2; w = 1.0; }
    else w = s - (double)j;
    const double* E = g_eff_Ed + i * EFF_NQ + j;
    const double E00 = __ldg(E), E01 = __ldg(E + 1), E10 = __ldg(E + EFF_NQ), E11 = __ldg(E + EFF_NQ + 1);
    const double e0 = E00 + w * (E01 - E00);
    const double e1 = E10 + w * (E11 - E10);
    return e0 + t * (e1 - e0);
}

// p of the gravitational kernel and its bound (err < 0: not applicable, use the exact sequence)
__device__ __forceinline__ void pair_prob_lite(double v1, double v2, uint64_t xmax, uint32_t n, double dt, double dv,
                                               double& p, double& err)
{
    err = -1.0;
    p = 0.0;
    const double vmin = fmin(v1, v2), vmax = fmax(v1, v2);
    if (!(vmin >= 0x1p-110) || !(vmax <= 0x1p+60) || !(dv >= 0x1p-100) || !(dv <= 0x1p+100)) return;
    const double r1 = cbrt_lite(__dmul_rn(v1, THREE_OVER_FOUR_PI)), r2 = cbrt_lite(__dmul_rn(v2, THREE_OVER_FOUR_PI));
    const double vt1 = vt_lite(r1), vt2 = vt_lite(r2);
    const double R = fmax(r1, r2), rs = fmin(r1, r2);
    const double E = efficiency_lite(R, rs * rcp_lite(R));
    const double sr = r1 + r2;
    const double a = PI_D * (sr * sr);
    const double scale = ((double)xmax * (double)(n - 1u + (n & 1u))) * (dt * rcp_lite(dv));
    p = ((a * fabs(vt1 - vt2)) * E) * scale;
    err = ((a * (vt1 + vt2)) * scale) * LITE_REL_BOUND + 0x1p-1000;
}

// gamma~ from the second filter; false when the interval does not settle it
__device__ __noinline__ bool gamma_tilde_lite(double v1, double v2, uint32_t n, double dt, double dv, uint64_t u53,
                                              uint64_t xi_j, uint64_t xi_k, uint64_t* g)
{
    double p, err;
    pair_prob_lite(v1, v2, xi_j, n, dt, dv, p, err);
    if (!(err >= 0.0) || !(p >= 0.0)) return false;
    const double lo = fmax(__dsub_rd(p, err), 0.0), hi = __dadd_ru(p, err);
    if (!(hi < 0x1p52)) return false;
    // floors of non-negative doubles below 2^52 by a round-down add of 2^52
    const double fl = __dsub_rn(__dadd_rd(lo, 0x1p52), 0x1p52);
    if (__dsub_rn(__dadd_rd(hi, 0x1p52), 0x1p52) != fl) {
        const uint64_t cap = xi_j / xi_k;
        if (fl >= 1.0 && (uint64_t)fl >= cap) { *g = cap; return true; }   // floor(p) >= floor(lo) >= cap
        return false;
    }
    const double phi = (double)u53 * 0x1p-53;      // exact
    uint64_t d;
    if (phi < lo - fl) d = 1;                      // phi < frac(p)   (lo - fl, hi - fl are exact)
    else if (phi >= hi - fl) d = 0;                // phi >= frac(p)
    else return false;
    const uint64_t gam = (uint64_t)fl + d;
    const uint64_t cap = gam <= 1 ? gam : xi_j / xi_k;
    *g = gam < cap ? gam : cap;
    return true;
}

// ---------------------------------------------------------------------------
// FP32 path with error bound
// ---------------------------------------------------------------------------
// Conversions to float are done with integer operations: on B300 the
// double->float and 64-bit integer->float conversion instructions issue on the
// (narrow) FP64 pipe.  Both helpers truncate the mantissa, so the result is
// within 2^-23 relative of the input (exact when the input fits 24 bits).

// |x| in [2^-126, 2^128): truncated float; smaller magnitudes give 0, larger +-inf.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - (1023 - 127);
    const uint32_t sign = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

__device__ __forceinline__ float u64_to_f_trunc(uint64_t x)
{
    if (x == 0) return 0.f;
    const int lz = __clzll((long long)x);
    const uint64_t n = x << lz;                       // leading one at bit 63
    return __uint_as_float(((uint32_t)(127 + 63 - lz) << 23) | ((uint32_t)(n >> 40) & 0x7fffffu));
}

// floor of a float >= 2^23 (such floats are integers), from its bits; saturates at
// 2^64 - 1 (infinity and NaN included).
__device__ __forceinline__ uint64_t f2u64_int(float x)
{
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    if (e >= 64 || (b >> 31)) return ~0ull;
    const uint64_t m = (uint64_t)((b & 0x7fffffu) | 0x800000u);
    return e >= 23 ? m << (e - 23) : m >> (23 - e);
}

// phi = u53 * 2^-53 lies in [t, t + 2^-23) with t = (u53 >> 30) * 2^-23; t is built
// exactly from bits as (1 + t) - 1.
__device__ __forceinline__ void phi_bounds23(uint64_t u53, float& lo, float& hi)
{
    const uint32_t t23 = (uint32_t)(u53 >> 30);
    lo = __uint_as_float(0x3F800000u | t23) - 1.0f;
    hi = lo + 0x1p-23f;
}

struct P32 { float p; float err; };

// Relative bound of the Golovin evaluation: five truncating conversions
// (v1, v2, xi, and the per-cell dt, dV: <= 2u each, u = 2^-24) and seven
// rounded FP32 operations give |p32 - p| <= 18 u p; 2^-17 = 128 u leaves a
// sevenfold margin.
constexpr float GOLOVIN_REL_BOUND = 0x1p-17f;
// Bound of the gravitational evaluation relative to
// B = scale * pi (r1+r2)^2 (vt1 + vt2) >= p / E (E <= 1), u = 2^-24:
//  r: truncated v (2u), 3/(4pi) (u), product (u), cbrtf (1 ulp = 2u) -> 3.4u;
//  vt: k r^2 law 9.8u, plus up to 4.4u where FP32 and FP64 pick different
//      regimes next to a (continuous) border -> 14.2u; so the difference
//      vt1 - vt2 is off by at most 15.2u (vt1 + vt2) in absolute terms;
//  pi (r1 + r2)^2: 11.8u;  scale (xi, S, dt/dV): 9u;
//  E: the interpolation weight along R is off by <= 28.4u (the radius nodes
//     satisfy R[i+1] / (R[i+1] - R[i]) <= 6), along q by <= 86u, times table
//     steps <= 1 and <= 0.2, plus roundings -> |dE| <= 52u absolute;
// in all |p32 - p64| <= (15.2 + 52 + 23.8) u B = 91u B (the FP64 value's own
// rounding is ~1e-14 relative).  2^-15 = 512u leaves a 5.6-fold margin.
constexpr float GRAV_REL_BOUND = 0x1p-15f;
constexpr float ABS_SLACK = 0x1p-100f;   // covers gradual underflow of the last products
constexpr float MIN_NORMAL_V = 0x1p-120f; // smaller float volumes are sent to the FP64 path

__device__ __forceinline__ float vt_f(float r)
{
    const float k1 = (float)VT_K1, k2 = (float)VT_K2, k3 = (float)VT_K3;
    const float r12 = (float)(VT_K2 / VT_K1);
    const float r23 = (float)((VT_K3 / VT_K2) * (VT_K3 / VT_K2));
    if (r < r12) return k1 * r * r;
    if (r < r23) return k2 * r;
    return k3 * sqrtf(r);
}

// FP32 copy of the efficiency table, staged in shared memory by every CTA that
// evaluates the gravitational kernel (divergent lookups into __constant__
// memory would serialise per distinct address).
struct EffTab {
    float R[EFF_NR];          // radius nodes
    float inv_dR[EFF_NR];     // 1 / (R[i+1] - R[i])
    float E[EFF_NR * EFF_NQ];
};

// the same table in global memory, for kernels that read it through L1 instead of staging it
__device__ const EffTab g_eff_tab = {
    {SDM_EFF_RADII(SDM_AS_FLOAT)},
    {SDM_INV_DR(0), SDM_INV_DR(1), SDM_INV_DR(2), SDM_INV_DR(3), SDM_INV_DR(4), SDM_INV_DR(5), SDM_INV_DR(6),
     SDM_INV_DR(7), SDM_INV_DR(8), SDM_INV_DR(9), SDM_INV_DR(10), 0.f},
    {SDM_EFF_VALUES(SDM_AS_FLOAT)}};

__device__ __forceinline__ void load_eff_tab(EffTab* T)
{
    for (int k = threadIdx.x; k < EFF_NR * EFF_NQ; k += blockDim.x) T->E[k] = c_eff_Ef[k];
    if (threadIdx.x < EFF_NR) {
        T->R[threadIdx.x] = c_eff_Rf[threadIdx.x];
        T->inv_dR[threadIdx.x] = c_eff_invdRf[threadIdx.x];
    }
}

__device__ __forceinline__ float efficiency_f(const EffTab* __restrict__ T, float R, float q)
{
    int i;
    float t;
    if (R <= 10e-6f) { i = 0; t = 0.f; }
    else if (R >= 1000e-6f) { i = EFF_NR - 2; t = 1.f; }
    else {
        // interval index by comparisons against the (uniform) node values
        i = (R >= 20e-6f) + (R >= 30e-6f) + (R >= 40e-6f) + (R >= 50e-6f) + (R >= 60e-6f) + (R >= 80e-6f) +
            (R >= 100e-6f) + (R >= 150e-6f) + (R >= 200e-6f) + (R >= 300e-6f);
        t = (R - T->R[i]) * T->inv_dR[i];
    }
    const float s = q * 10.f;
    const float sf = __fadd_rd(s, 0x1p23f);               // 2^23 + floor(s), exact for 0 <= s < 2^23
    int j = (int)(__float_as_uint(sf) - 0x4B000000u);
    float w;
    if (j >= EFF_NQ - 1) { j = EFF_NQ - 2; w = 1.f; }
    else w = s - (sf - 0x1p23f);
    const float* E = T->E + i * EFF_NQ + j;
    const float e0 = E[0] + w * (E[1] - E[0]);
    const float e1 = E[EFF_NQ] + w * (E[EFF_NQ + 1] - E[EFF_NQ]);
    return e0 + t * (e1 - e0);
}

// E together with a bound dE on |E - E_exact| (absolute), E_exact the efficiency of the
// exact radii (u = 2^-24): the interpolation weight along q is off by at most
// 10 * 8u * q (radii 3.4u each, the division and the scaling by 10), along R by at
// most 4.4u R / dR + 2u; the weights multiply the table steps actually used, and the
// roundings of the interpolation and of the float copy of the table add at most 12u.
// dE < 0 when R or 10 q lies too close to a table node for the interval to be certain
// (the caller then uses the pair-independent bound).
__device__ __forceinline__ float efficiency_f_err(const EffTab* __restrict__ T, float R, float q, float& dE)
{
    const float u = 0x1p-24f;
    int i;
    float t, dt;
    bool near = false;
    if (R <= 10e-6f) { i = 0; t = 0.f; dt = 0.f; near = R >= 10e-6f * (1.0f - 8.0f * u); }
    else if (R >= 1000e-6f) { i = EFF_NR - 2; t = 1.f; dt = 0.f; near = R <= 1000e-6f * (1.0f + 8.0f * u); }
    else {
        i = (R >= 20e-6f) + (R >= 30e-6f) + (R >= 40e-6f) + (R >= 50e-6f) + (R >= 60e-6f) + (R >= 80e-6f) +
            (R >= 100e-6f) + (R >= 150e-6f) + (R >= 200e-6f) + (R >= 300e-6f);
        t = (R - T->R[i]) * T->inv_dR[i];
        dt = (4.4f * u) * (R * T->inv_dR[i]) + 2.0f * u;
        near = t <= 2.0f * dt || t >= 1.0f - 2.0f * dt;
    }
    const float s = q * 10.f;
    const float sf = __fadd_rd(s, 0x1p23f);
    int j = (int)(__float_as_uint(sf) - 0x4B000000u);
    float w;
    if (j >= EFF_NQ - 1) { j = EFF_NQ - 2; w = 1.f; }
    else w = s - (sf - 0x1p23f);
    const float dw = (80.0f * u) * q + (10.0f * u) * q;
    near = near || w <= 2.0f * dw || (j < EFF_NQ - 2 && w >= 1.0f - 2.0f * dw);
    const float* E = T->E + i * EFF_NQ + j;
    const float d0 = E[1] - E[0], d1 = E[EFF_NQ + 1] - E[EFF_NQ];
    const float e0 = E[0] + w * d0;
    const float e1 = E[EFF_NQ] + w * d1;
    const float Dw = fmaxf(fabsf(d0), fabsf(d1)), Dt = fabsf(e1 - e0) + 4.0f * u;
    dE = near ? -1.0f : Dw * dw + Dt * dt + 12.0f * u;
    return e0 + t * (e1 - e0);
}

// p in FP32 with its bound.  scale32 = max(xi) * S_c * dt / dV in FP32; efield_f the electric-field
// kernel's field parameter rounded to float.  A non-finite or NaN err marks the pair for the FP64
// path.
__device__ __forceinline__ P32 pair_prob_f(const EffTab* __restrict__ T, uint32_t kid, double v1d, double v2d,
                                           float scale32, float golovin_bf, float efield_f = 0.0f)
{
    const float v1 = d2f_trunc(v1d), v2 = d2f_trunc(v2d);
    P32 o;
    if (!(fminf(v1, v2) >= MIN_NORMAL_V)) { o.p = 0.f; o.err = __int_as_float(0x7fc00000); return o; }
    if (kid == 0) {
        const float K = golovin_bf * (v1 + v2);
        o.p = K * scale32;
        o.err = o.p * GOLOVIN_REL_BOUND + ABS_SLACK;
        return o;
    }
    const float c = (float)THREE_OVER_FOUR_PI;
    const float r1 = cbrtf(v1 * c), r2 = cbrtf(v2 * c);
    const float vt1 = vt_f(r1), vt2 = vt_f(r2);
    const float R = fmaxf(r1, r2), rs = fminf(r1, r2);
    float dE;
    float E = efficiency_f_err(T, R, rs / R, dE);
    if (kid == 2) {
        // E_eps = E + eps (1 - E): the error of E passes times 1 - eps <= 1; the three roundings
        // and the rounding of eps add at most 4u (u = 2^-24; E_eps <= 1), so dE + 5u bounds it
        E = E + efield_f * (1.0f - E);
        if (dE >= 0.0f) dE += 5.0f * 0x1p-24f;
    }
    const float s = r1 + r2;
    const float base = scale32 * ((float)PI_D * (s * s));
    const float dvt = fabsf(vt1 - vt2), svt = vt1 + vt2;
    o.p = (base * dvt) * E;
    if (dE >= 0.0f) {
        // Pair-specific bound (u = 2^-24), relative to base = scale pi (r1+r2)^2:
        //  scale (9u), (r1+r2)^2 with radii within 3.4u (9.8u), pi and the products (4u) and
        //  the final roundings: |dvt| E 25u;  fall speeds within 15u of the exact ones
        //  (regime choice included), so |dvt| is off by 15u (vt1 + vt2) absolute: E 15u svt;
        //  the efficiency: |dvt| dE;  the exact sequence's own error: 2^-45 svt.
        // Doubled, and 64u more for evaluating it from the rounded base.
        const float u = 0x1p-24f;
        const float e = dvt * (25.0f * u * E + dE) + svt * (15.0f * u * E + 0x1p-45f);
        o.err = (base * e) * (2.0f + 128.0f * u) + ABS_SLACK;
    } else {
        o.err = (base * svt) * GRAV_REL_BOUND + ABS_SLACK;
    }
    return o;
}

// Decide gamma~ from the FP32 interval.  Returns true when settled (result in
// *g), false when the FP64 path must decide.
__device__ __forceinline__ bool gamma_tilde_certified(P32 pe, uint64_t u53, uint64_t xi_j, uint64_t xi_k,
                                                      uint64_t* g)
{
    float lo = __fsub_rd(pe.p, pe.err);
    const float hi = __fadd_ru(pe.p, pe.err);
    if (!(hi < 0x1p23f) || !(lo == lo)) {
        // large, non-finite or NaN: only a binding cap can settle it here
        if (lo >= 0x1p23f && lo == lo) {
            const uint64_t cap = xi_j / xi_k;
            if (f2u64_int(lo) >= cap) { *g = cap; return true; }   // floor(p) >= lo >= cap
        }
        return false;
    }
    lo = fmaxf(lo, 0.f);
    // floors of lo and hi (both in [0, 2^23)) from the bits of x + 2^23 rounded down;
    // no float<->int conversion instruction is used (on B300 they issue on the FP64 pipe)
    const float tl = __fadd_rd(lo, 0x1p23f), th = __fadd_rd(hi, 0x1p23f);
    const uint32_t m = __float_as_uint(tl) - 0x4B000000u;      // floor(lo)
    if (tl != th) {
        if (m >= 1u) {
            const uint64_t cap = xi_j / xi_k;
            if ((uint64_t)m >= cap) { *g = cap; return true; }
        }
        return false;
    }
    // floor(p) = m is certain; frac(p) lies in [lo - m, hi - m] (both exact)
    const float fl = tl - 0x1p23f;
    const float f_lo = lo - fl, f_hi = hi - fl;
    float phi_lo, phi_hi;
    phi_bounds23(u53, phi_lo, phi_hi);
    uint32_t d;
    if (phi_hi <= f_lo) d = 1;          // phi < phi_hi <= frac
    else if (phi_lo >= f_hi) d = 0;     // phi >= phi_lo >= frac
    else return false;
    const uint32_t gam = m + d;
    if (gam <= 1u) { *g = gam; return true; }      // xi_j >= xi_k so the cap is >= 1
    const uint64_t cap = xi_j / xi_k;
    *g = (uint64_t)gam < cap ? (uint64_t)gam : cap;
    return true;
}

// ---------------------------------------------------------------------------
// Early exit of Step 3: an upper bound of p from the bins of the pair's two
// volumes and its larger multiplicity.  When phi >= bound >= p (and so p < 1),
// gamma = floor(p) + [phi < p] = 0 and the pair needs no kernel evaluation.
// The bound holds for the FP64 value and for the FP32 value alike.
//   bin of a volume v: its double exponent e and two leading mantissa bits m,
//   bin = 4 (e - PB_EMIN) + m covering [2^e (1 + m/4), 2^e (1 + (m+1)/4));
//   volumes below the first bin join it (its lower edge is 0), volumes above
//   the last have no bound.
//   table[kind][b1][d]: b1 the larger volume's bin, d = b1 - b2 the distance to
//   the smaller one's, the last column (d = PB_ND) for every b2 <= b1 - PB_ND
//   (smaller volume anywhere in [0, upper edge of bin b1 - PB_ND)):
//     Golovin: the sum of the two upper edges (K = b (v1 + v2));
//     gravitational: pi (R+ + r+)^2 (vt(R+) - vt(r-) + 2^-12 (vt(R+) + vt(r+)))
//     Emax (electric field: Emax = 1, the bound of E_eps for every field parameter),
//     with R+- and r+- the radii at the bins' edges (vt grows with the
//     radius, so |vt1 - vt2| <= vt(R+) - vt(r-); the 2^-12 term covers the
//     FP32 path's error, which is relative to vt1 + vt2) and Emax the largest
//     value of the interpolated efficiency for R in [R-, R+], q = r/R in
//     [r-/R+, min(1, r+/R-)] (bilinear on each table cell, so taken at the
//     rectangle's corners and where node lines cut its edges or cross inside);
//   times 1 + 2^-10, rounded up to float.  Filled by the host once per device.
//   p <= table * c_up * X with c_up = S dt/dV (* b for Golovin) * (1 + 2^-8)
//   rounded up and X >= max(xi1, xi2) -- per pair the power of two
//   2^(64 - clz(xi1 | xi2)), or per cell its largest multiplicity rounded up
//   to float, which stays valid for every later step because coalescence
//   never raises a multiplicity; the margins cover the FP32 scale's roundings
//   and the FP32 path's own error.
// ---------------------------------------------------------------------------
constexpr int PB_EMIN = -80;
constexpr uint32_t PB_NB = 255;                                  // exponents -80 .. -17 (a bin fits a byte)
constexpr uint32_t PB_HI0 = (uint32_t)(1023 + PB_EMIN) << 2;      // (high word >> 18) of bin 0
constexpr uint32_t PB_ND = 32;                                    // bin distances 0 .. PB_ND - 1, then the rest
constexpr uint32_t PB_ROW = PB_ND + 1;
constexpr uint32_t PB_SIZE = (PB_NB + 1) * PB_ROW;                // row PB_NB: +inf
constexpr uint32_t PB_KINDS = 3;                                  // Golovin, gravitational, electric field
__device__ float g_pbound[PB_KINDS][PB_SIZE];

// Early-exit key of a volume: the top 14 bits of its high word (sign, exponent, two
// mantissa bits).  Non-negative doubles order as their keys.
__device__ __forceinline__ uint32_t vkey_of(double v)
{
    return (uint32_t)__double2hiint(v) >> 18;
}

// bin of a non-negative volume from its key (PB_NB: beyond the table)
__device__ __forceinline__ uint32_t pb_bin_key(uint32_t k)
{
    return k < PB_HI0 ? 0u : min(k - PB_HI0, PB_NB);
}

__device__ __forceinline__ uint32_t vbin_of(double v)
{
    return pb_bin_key(vkey_of(v));
}

// entry of the bound table for two volumes' bins
__device__ __forceinline__ uint32_t pb_index(uint32_t b1, uint32_t b2)
{
    const uint32_t hi = max(b1, b2);
    return hi * PB_ROW + min(hi - min(b1, b2), PB_ND);
}

// 2^(64 - clz(x1 | x2)) > max(x1, x2) as a float (x1 | x2 != 0, both < 2^53)
__device__ __forceinline__ float xi_pow2_above(uint64_t x1, uint64_t x2)
{
    const uint32_t lz = (uint32_t)__clzll((long long)(x1 | x2));
    return __uint_as_float((127u + 64u - lz) << 23);
}

// phi's leading 23 bits as a float phi_lo <= phi; w_hi = the high Philox word of the pair's phi
__device__ __forceinline__ float phi_lo23(uint32_t w_hi)
{
    return __uint_as_float(0x3F800000u | (w_hi >> 9)) - 1.0f;
}

// FP32 mode: gamma from p32 and the leading 23 bits of phi.
__device__ __forceinline__ uint64_t gamma_tilde_f(float p, uint64_t u53, uint64_t xi_j, uint64_t xi_k)
{
    if (!(p < 0x1p23f)) {
        const uint64_t cap = xi_j / xi_k;
        const uint64_t gam = f2u64_int(p);          // floats >= 2^23 are integers
        return gam < cap ? gam : cap;
    }
    const float t = __fadd_rd(p, 0x1p23f);
    const uint32_t fl = __float_as_uint(t) - 0x4B000000u;
    const float frac = p - (t - 0x1p23f);
    float phi_lo, phi_hi;
    phi_bounds23(u53, phi_lo, phi_hi);
    const uint32_t gam = fl + (phi_lo < frac ? 1u : 0u);
    if (gam <= 1u) return gam;
    const uint64_t cap = xi_j / xi_k;
    return (uint64_t)gam < cap ? (uint64_t)gam : cap;
}

}  // namespace sdm
