// Device-side data structures and per-cell physics of the reacting-flow RHS.
//
// Every function here is templated on R, the type of the bulk arithmetic
// (double for the FP64 path, float for the mixed path), and on NS, the species
// count, so that species loops unroll into registers.  The parts the mixed
// path keeps in FP64 are written with double explicitly: the temperature
// Newton solve, the Gibbs energies, equilibrium constants and reverse rates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rf {

constexpr int NSMAX = 9;
constexpr int NRMAX = 32;
constexpr int NPMAX = 8;                  // pressure-dependent reactions per mechanism
constexpr double RU = 8.314462618;    // J/mol/K
constexpr double PATM = 101325.0;     // Pa
constexpr double EPS_WENO = 1.0e-30;
constexpr double EPS_D = 1.0e-12;
constexpr double T_MAX_ADMISSIBLE = 1.0e5;

enum StatusBits : int { ST_NEWTON = 1, ST_NONFINITE = 2, ST_RANGE = 4, ST_TIMEOUT = 8 };

// Mechanism constants (species, NASA-7 sets, transport, compact reactions).
struct MechDev {
    int ns, nr, two_ranges, npress;            // npress: pressure-dependent reactions
    double Tmid;
    double W[NSMAX], invW[NSMAX], RW[NSMAX];   // R/W_s
    double cpc[2][NSMAX][5];                   // cp/R = c0 + c1 T + ... + c4 T^4, per range
    double ec[2][NSMAX][6];                    // a1, a2/2, a3/3, a4/4, a5/5, a6 (h/RT Horner + a6/T)
    double ecR[2][NSMAX][6];                   // e_s / T-powers: (a1 - 1) R/W_s, then ec times R/W_s (Newton solve)
    double gc[2][NSMAX][7];                    // ln G = g/RT + ln(RT/p_atm) = gc0 + T(gc1 + ... T gc4) + gc5/T + gc6 lnT
    double gc0w[2][NSMAX];                     // gc0 - ln W_s: ln (G_s / W_s), the mixed path's Gibbs factor
    float ecf[2][NSMAX][6];                    // FP32 copy of ec
    double mu_ref[NSMAX], mu_exp[NSMAX], eucken[NSMAX];     // eucken = 1.25 R / W_s
    double hl_mu_ref[NSMAX], h_mu_exp[NSMAX];  // ln(mu_ref) / 2, mu_exp / 2: sqrt(mu_s) by one exponential
    double invDref[NSMAX][NSMAX];
    double wc[NSMAX][NSMAX];                   // (W_j / W_i)^(1/4)
    double wd[NSMAX][NSMAX];                   // 1 / sqrt(8 (1 + W_i / W_j))
    float Wf[NSMAX], invWf[NSMAX], RWf[NSMAX];
    float cpcf[2][NSMAX][5];
    float mu_reff[NSMAX], mu_expf[NSMAX], euckenf[NSMAX];
    float invDreff[NSMAX][NSMAX];
    float wcf[NSMAX][NSMAX], wdf[NSMAX][NSMAX];
    // reactions: compact stoichiometry (species indices repeated by coefficient)
    double lnA[NRMAX], A[NRMAX], b[NRMAX], Theta[NRMAX];
    float lnAf[NRMAX], bf[NRMAX], Thetaf[NRMAX];
    int8_t n_reac[NRMAX], n_prod[NRMAX], reac[NRMAX][3], prod[NRMAX][3];
    int8_t n_net[NRMAX], net_sp[NRMAX][6], net_nu[NRMAX][6];
    int8_t dnu_sum[NRMAX], rev[NRMAX];
    // factors of the reverse term k_f prod_prod (C G)_s prod_reac (1/G)_s: products
    // (species s) then reactants (s + 16), in that order
    int8_t n_revf[NRMAX], revf[NRMAX][6];
    // net coefficient nu''_s - nu'_s of the species at each reactant / product position
    int8_t dnu_reac[NRMAX][3], dnu_prod[NRMAX][3];
    // pressure-dependent reactions: ptype 0 elementary, 1 third body, 2 Lindemann,
    // 3 Troe fall-off; pslot indexes the tables below (efficiencies of [M], the
    // low-pressure Arrhenius ln A0, b0, Theta0, Troe alpha, T***, T*, T**)
    int8_t ptype[NRMAX], pslot[NRMAX];
    // reactions grouped by shape for the mixed path's rate-of-progress pass: classes
    // 0..3 are reversible elementary reactions with (1, 1), (1, 2), (2, 1), (2, 2)
    // reactant and product molecules, class 4 everything else; cls_rx[cls_start[c] ..
    // cls_start[c + 1]) lists the reactions of class c
    int8_t cls_start[6], cls_rx[NRMAX];
    // species-major lists of the net coefficients (reactions ascending): species s
    // takes nu = sp_nu[e] times q of reaction sp_rx[e] for e in [sp_start[s], sp_start[s + 1])
    int16_t sp_start[NSMAX + 1];
    int8_t sp_rx[NRMAX * 6], sp_nu[NRMAX * 6];
    float kapf[NRMAX];                         // prod over reactant molecules of 1 / W_s (mixed path)
    double eff[NPMAX][NSMAX], lnA0[NPMAX], b0[NPMAX], Theta0[NPMAX], troe[NPMAX][4];
    float efff[NPMAX][NSMAX], lnA0f[NPMAX], b0f[NPMAX], Theta0f[NPMAX], troef[NPMAX][4];
};

// Mechanisms in use live in constant-memory slots; kernels receive the slot
// index, so their constants are read through the constant cache and graph
// nodes carry no large parameter block.
constexpr int MECH_SLOTS = 5;             // 5 x sizeof(MechDev) within the 64 KB constant bank
__constant__ MechDev c_mech[MECH_SLOTS];

// One grid and the buffers of one evaluation or RK stage.
struct Member {
    int nx, ny, nz;
    int bc[3];
    double h[3], invh[3];
    double weps[3];              // h^2 / 3 per axis: the WENO3-Z eps is weps (a^2 + b^2 + c^2) + EPS_WENO
    long long n;                 // cells
    const double *U;             // stage input state (FP64, [nv][n])
    const double *Un;            // state at the start of the step (stage update)
    double *Uout;                // stage output state (FP64)
    double *dUdt;                // rf_rhs output (FP64)
    double *T;                   // temperature warm start in/out
    void *Q;                     // primitive/coefficient fields, type R
    void *rhs;                   // RHS accumulator, type R
    float *U32;                  // FP32 copy of U (mixed path)
    double *clock;               // [0] = t, [1] = dt, [2] = CFL, [3] = dt_fixed (<= 0: rule)
    unsigned long long *rates;   // [0] acoustic, [1] diffusive, [2] chemical maxima (double bits)
    int *status;
    long long *bad_cell;
    double stage_a, stage_b, stage_c;   // U_out = a Un + b (U + dt L), time t + c dt
    double las[7];               // E, x0, y0, z0, sigma_r, t0, sigma_t
    double las_k[3];             // E / ((2 pi)^2 sigma_r^3 sigma_t) (nz = 1: E / ((2 pi)^(3/2) sigma_r^2 sigma_t)),
                                 // -1 / (2 sigma_r^2), 1 / sigma_t
    double las_c0[3];            // centre of cell 0 minus x0, y0, z0
    int laser_on;
    int flags;
    int want_rates;
    int t_from_host;             // 1: stage time is t_host (rf_rhs), 0: clock[0] + stage_c clock[1]
    double t_host;
    int xW, xrpb;                // x sweep row chunk width and rows per block (ensemble launches)
    long long c_lo, c_hi;        // cells [c_lo, c_hi) of a cell-state launch
    // mapped grids (null on Cartesian ones): face area vectors per axis [3][faces of
    // the axis], cell metric d xi_e / d x_k [9][n] and 1/volume [n] (all of type R),
    // cell volume [n] and centres [3][n] (FP64)
    int mapped;
    const void *gS[3];
    const void *gM, *giV;
    const double *gV, *gC;
};

// Q field order (each field n values of type R).
enum QField { Q_U = 0, Q_V = 1, Q_W = 2, Q_P = 3, Q_C = 4, Q_T = 5, Q_MU = 6, Q_LAM = 7, Q_X0 = 8 };
template <int NS> struct QL {
    static constexpr int X = Q_X0, DC = Q_X0 + NS, H = Q_X0 + 2 * NS, NQ = Q_X0 + 3 * NS;
};


// ----------------------------------------------------------------------------- binary32 <-> binary64

// Conversions between IEEE 754 binary32 and binary64 from integer operations on the bit
// fields.  The hardware conversions execute on the FP64 unit at its rate, and the FP64
// unit is what bounds the mixed-precision cell state; these run on the integer pipes,
// every input class included (a hardware conversion kept for the rare classes was
// still issued, predicated off, on the common path).  The rare classes sit in
// functions of their own, so the common path is a test and a branch (zeros, common
// in the species fields, are handled inline).  Both return what
// the hardware conversion (round to nearest even, subnormals kept) returns for every
// non-NaN input; a NaN converts to a quiet NaN with the same sign and the leading
// payload bits.

// binary32 -> binary64 (exact).  Normal numbers: the 8-bit exponent is rebiased
// (127 -> 1023) and the 23 mantissa bits become the top of the 52; zeros keep their
// sign; a subnormal a 2^-149 is normalised at its leading bit.
__device__ __noinline__ double f2d_rare(unsigned u) {
    const unsigned a = u & 0x7fffffffu, sg = u & 0x80000000u;
    if (a == 0u) return __hiloint2double((int)sg, 0);
    if (a >= 0x7f800000u)                            // infinity, or NaN (quieted)
        return __hiloint2double((int)(sg | 0x7ff00000u | (a == 0x7f800000u ? 0u : 0x00080000u) | ((a & 0x7fffffu) >> 3)),
                                (int)(a << 29));
    const int lz = __clz(a);                         // 9 .. 31: leading bit at 31 - lz, value 2^(-118 - lz) (1.f)
    const unsigned f = (a << lz) << 1;               // fraction bits below it, left-aligned
    return __hiloint2double((int)(sg | ((unsigned)(905 - lz) << 20) | (f >> 12)), (int)(f << 20));
}
__device__ __forceinline__ double f2d(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned a = u & 0x7fffffffu;
    if (a - 0x00800000u >= 0x7f000000u) {            // zero, subnormal, infinity or NaN
        if (a == 0u) return __hiloint2double((int)u, 0);
        return f2d_rare(u);
    }
    return __hiloint2double((int)(((a >> 3) + (896u << 20)) | (u & 0x80000000u)), (int)(a << 29));
}

// binary64 -> binary32, round to nearest even.  For 2^-126 <= |x| < 2^128 the exponent
// is rebiased (1023 -> 127), the top 23 of the 52 mantissa bits are kept and the 29
// below them rounded; a carry out of the mantissa is the next binade (or infinity),
// as in IEEE rounding.  Below 2^-126 the 53-bit significand is shifted onto the
// subnormal grid (2^-149) and rounded the same way (|x| <= 2^-150 gives a signed
// zero); from 2^128 on the result is infinity.
__device__ __noinline__ float d2f_rare(unsigned hi, unsigned lo) {
    const unsigned e = (hi >> 20) & 0x7ffu, sg = hi & 0x80000000u;
    if (e >= 1151u) {                                // |x| >= 2^128, infinity or NaN
        const bool nan = e == 2047u && ((hi & 0xfffffu) | lo) != 0u;
        return __uint_as_float(sg | 0x7f800000u | (nan ? 0x00400000u | ((hi & 0xfffffu) << 3) | (lo >> 29) : 0u));
    }
    if (e < 873u) return __uint_as_float(sg);        // |x| < 2^-150
    const unsigned long long M = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
    const unsigned sh = 926u - e;                    // 30 .. 53: M 2^(e - 1075) = (M >> sh) 2^-149
    const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
    const unsigned r = (unsigned)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
    return __uint_as_float(sg | r);
}
__device__ __forceinline__ float d2f(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u >= 254u) {                          // outside [2^-126, 2^128)
        if (e < 873u) return __uint_as_float(hi & 0x80000000u);   // |x| < 2^-150 (zero included)
        return d2f_rare(hi, lo);
    }
    // (hi:lo) << 3: the low nine exponent bits and the top 23 mantissa bits; the
    // rebias 1023 -> 127 is -896 = -384 (mod 512) in the nine-bit exponent field
    unsigned t = __funnelshift_l(lo, hi, 3) - (384u << 23);
    const unsigned rem = lo & 0x1fffffffu;           // the 29 bits rounded away
    t += (rem + (t & 1u)) > 0x10000000u ? 1u : 0u;   // above half, or half and odd
    return __uint_as_float(t | (hi & 0x80000000u));
}

// Comparisons of doubles on their bit patterns (integer pipes): non-negative doubles
// order like their patterns, and an exponent field of all ones is an infinity or a NaN.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool finite64(double x) { return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u; }
// 0 < x < b, for a positive finite bound b (false for zero, negative, infinite and NaN x)
__device__ __forceinline__ bool in_open_pos(double x, double b) {
    return (unsigned long long)(dbits(x) - 1) < (unsigned long long)(dbits(b) - 1);
}
// |x| <= b, for b >= 0 (false for NaN x)
__device__ __forceinline__ bool abs_le(double x, double b) {
    return (unsigned long long)(dbits(x) & 0x7fffffffffffffffll) <= (unsigned long long)dbits(b);
}
// x >= b, for b > 0 and x not NaN
__device__ __forceinline__ bool ge_pos(double x, double b) { return dbits(x) >= dbits(b); }

// FP64 value of a bulk-type number and bulk-type value of an FP64 number.
__device__ __forceinline__ double wide(float x) { return f2d(x); }
__device__ __forceinline__ double wide(double x) { return x; }
template <typename R> __device__ __forceinline__ R narrow(double x);
template <> __device__ __forceinline__ float narrow<float>(double x) { return d2f(x); }
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }

// 1/x in FP64 from an FP32 seed r (correctly rounded, |e| <= 2^-24 with e = 1 - x r,
// which one FMA gives exactly): 1/x = r / (1 - e) = r (1 + e + e^2 + ...), and
// r + r (e + e^2) leaves e^3 <= 2^-72 relative, below FP64 rounding.  For x whose
// magnitude lies in the FP32 normal range (densities, temperatures, gas constants).
__device__ __forceinline__ double rcp64(double x) {
    const double r = f2d(__frcp_rn(d2f(x)));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

template <typename R> __device__ __forceinline__ R mech_mu_ref(const MechDev &M, int s);
template <> __device__ __forceinline__ double mech_mu_ref<double>(const MechDev &M, int s) { return M.mu_ref[s]; }
template <> __device__ __forceinline__ float mech_mu_ref<float>(const MechDev &M, int s) { return M.mu_reff[s]; }
template <typename R> __device__ __forceinline__ R mech_mu_exp(const MechDev &M, int s);
template <> __device__ __forceinline__ double mech_mu_exp<double>(const MechDev &M, int s) { return M.mu_exp[s]; }
template <> __device__ __forceinline__ float mech_mu_exp<float>(const MechDev &M, int s) { return M.mu_expf[s]; }
template <typename R> __device__ __forceinline__ R mech_eucken(const MechDev &M, int s);
template <> __device__ __forceinline__ double mech_eucken<double>(const MechDev &M, int s) { return M.eucken[s]; }
template <> __device__ __forceinline__ float mech_eucken<float>(const MechDev &M, int s) { return M.euckenf[s]; }
template <typename R> __device__ __forceinline__ R mech_invD(const MechDev &M, int s, int j);
template <> __device__ __forceinline__ double mech_invD<double>(const MechDev &M, int s, int j) { return M.invDref[s][j]; }
template <> __device__ __forceinline__ float mech_invD<float>(const MechDev &M, int s, int j) { return M.invDreff[s][j]; }
template <typename R> __device__ __forceinline__ R mech_wc(const MechDev &M, int i, int j);
template <> __device__ __forceinline__ double mech_wc<double>(const MechDev &M, int i, int j) { return M.wc[i][j]; }
template <> __device__ __forceinline__ float mech_wc<float>(const MechDev &M, int i, int j) { return M.wcf[i][j]; }
template <typename R> __device__ __forceinline__ R mech_wd(const MechDev &M, int i, int j);
template <> __device__ __forceinline__ double mech_wd<double>(const MechDev &M, int i, int j) { return M.wd[i][j]; }
template <> __device__ __forceinline__ float mech_wd<float>(const MechDev &M, int i, int j) { return M.wdf[i][j]; }
template <typename R> __device__ __forceinline__ R mech_W(const MechDev &M, int s);
template <> __device__ __forceinline__ double mech_W<double>(const MechDev &M, int s) { return M.W[s]; }
template <> __device__ __forceinline__ float mech_W<float>(const MechDev &M, int s) { return M.Wf[s]; }
template <typename R> __device__ __forceinline__ R mech_RW(const MechDev &M, int s);
template <> __device__ __forceinline__ double mech_RW<double>(const MechDev &M, int s) { return M.RW[s]; }
template <> __device__ __forceinline__ float mech_RW<float>(const MechDev &M, int s) { return M.RWf[s]; }
template <typename R> __device__ __forceinline__ R mech_cpc(const MechDev &M, int r, int s, int k);
template <> __device__ __forceinline__ double mech_cpc<double>(const MechDev &M, int r, int s, int k) { return M.cpc[r][s][k]; }
template <> __device__ __forceinline__ float mech_cpc<float>(const MechDev &M, int r, int s, int k) { return M.cpcf[r][s][k]; }

// ----------------------------------------------------------------------------- exponential pair

// exp(x) and exp(-x) in FP64 from one argument reduction, after Tang's
// table-driven exponential (P. T. P. Tang, ACM TOMS 15 (1989) 144-157):
// x = k ln2/256 + r with k = 256 m + j, 0 <= j < 256, |r| <= ln2/512, and
//   exp(+-x) = 2^(+-m) 2^(+-j/256) (E(r) +- O(r)),
// E = 1 + r^2/2 + r^4/24 and O = r + r^3/6 the even and odd parts of the Taylor
// series of exp(r) (first omitted terms r^6/720 < 1e-20 and r^5/120 < 4e-17
// relative).  ln2/256 is split into its double value and the remainder so that r
// keeps full precision for every k; 2^(+-m) is added to the exponent fields of the
// correctly rounded table entries.  A few ulp from exp itself for |x| <= 707;
// for 707 < |x| < 45,000 the power of two is clamped to 2^(+-1020) and the results
// saturate.  The reduction is valid only while k = round(256 x / ln 2) converts
// exactly through FP32 (|k| < 2^24, i.e. |x| < 45,000); callers keep their
// arguments far inside that (Gibbs energies and Arrhenius exponents of a few
// hundred, the laser exponent bounded at -740).
constexpr double LN2_256_HI = 0.6931471805599453094 / 256.0;   // double(ln 2) / 256, exact
constexpr double LN2_256_LO = 2.3190468138462996e-17 / 256.0;  // (ln 2 - double(ln 2)) / 256
__device__ double g_exp_tab[512];                              // 2^(j/256), then 2^(-j/256), j = 0..255

__device__ __forceinline__ void exp_pair(double x, double &ep, double &em) {
    const double shifter = 6755399441055744.0;               // 1.5 * 2^52: rounds to an integer in the low bits
    const double t = fma(x, 369.3299304675746 /* 256 / ln 2 */, shifter);
    const int k = __double2loint(t);
    const double kd = f2d((float)k);                          // = t - shifter, exactly (|k| < 2^24)
    double r = fma(-kd, LN2_256_HI, x);
    r = fma(-kd, LN2_256_LO, r);
    const double r2 = r * r;
    const double E = fma(r2, fma(r2, 1.0 / 24.0, 0.5), 1.0);
    const double O = fma(r * r2, 1.0 / 6.0, r);
    const int j = k & 255, m = min(max(k >> 8, -1020), 1020);
    const double tp = __ldg(&g_exp_tab[j]), tm = __ldg(&g_exp_tab[256 + j]);
    const double sp = __hiloint2double(__double2hiint(tp) + (m << 20), __double2loint(tp));
    const double sm = __hiloint2double(__double2hiint(tm) - (m << 20), __double2loint(tm));
    ep = sp * (E + O);
    em = sm * (E - O);
}

// The mixed path's exponential pair.  Its Gibbs factors feed a reverse term that is
// subtracted from an FP32 forward term, so a relative error of 2e-13 loses nothing
// there.  The same reduction without the low part of ln2/256 (which moves r by at most
// |x| 3.4e-17), and exp(+-r) = 1 +- r + p(+-r) with the small part
// p(r) = r^2 (1/2 + r (1/6 + r/24)) <= 9.2e-7 formed in FP32 from r rounded to FP32
// (relative error about 1.2e-7, so at most 1.1e-13 absolute; the first omitted term
// r^5/120 < 4e-17): the FP64 work is the reduction and two FMAs per exponential,
// s (1 + p) then + s r, with the scale s the table entry.
__device__ __forceinline__ void exp_pair_mixed(double x, double &ep, double &em) {
    const double shifter = 6755399441055744.0;
    const double t = fma(x, 369.3299304675746 /* 256 / ln 2 */, shifter);
    const int k = __double2loint(t);
    const double kd = f2d((float)k);                          // = t - shifter, exactly (|k| < 2^24)
    const double r = fma(-kd, LN2_256_HI, x);
    const float rf = d2f(r), r2f = rf * rf;
    const float pp = r2f * fmaf(rf, fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
    const float pm = r2f * fmaf(-rf, fmaf(-rf, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
    const int j = k & 255, m = min(max(k >> 8, -1020), 1020);
    const double tp = __ldg(&g_exp_tab[j]), tm = __ldg(&g_exp_tab[256 + j]);
    const double sp = __hiloint2double(__double2hiint(tp) + (m << 20), __double2loint(tp));
    const double sm = __hiloint2double(__double2hiint(tm) - (m << 20), __double2loint(tm));
    ep = fma(sp, r, fma(sp, f2d(pp), sp));
    em = fma(-sm, r, fma(sm, f2d(pm), sm));
}

// exp(x) alone from the same reduction and table: exp(r) by its Taylor polynomial
// through r^4 (first omitted term r^5/120 < 4e-17 relative), one table factor.
__device__ __forceinline__ double exp64(double x) {
    const double shifter = 6755399441055744.0;
    const double t = fma(x, 369.3299304675746 /* 256 / ln 2 */, shifter);
    const int k = __double2loint(t);
    const double kd = f2d((float)k);                          // = t - shifter, exactly (|k| < 2^24)
    double r = fma(-kd, LN2_256_HI, x);
    r = fma(-kd, LN2_256_LO, r);
    const double p = fma(r, fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0), 1.0);
    const int j = k & 255, m = min(max(k >> 8, -1020), 1020);
    const double tp = __ldg(&g_exp_tab[j]);
    return __hiloint2double(__double2hiint(tp) + (m << 20), __double2loint(tp)) * p;
}

// ----------------------------------------------------------------------------- logarithm

// ln x in FP64 for normal x > 0, after Tang's table-driven logarithm (P. T. P. Tang,
// ACM TOMS 16 (1990) 378-400): x = 2^m y with y in [1, 2), F = 1 + j/64 the nearest
// table point (from the leading mantissa bits, exact), f = y - F (exact),
// r = f / F (|r| <= 1/128) and
//   ln x = m ln2 + ln F + ln(1 + r),  ln(1 + r) = r - r^2/2 + ... - r^6/6
// (first omitted term r^7/7 < 4e-17).  ln 2 and ln F are carried as high and low
// parts; 1/F and ln F are tabulated from extended precision.
constexpr double LN2_HI = 0.6931471805599453094;           // double(ln 2)
constexpr double LN2_LO = 2.3190468138462996e-17;          // ln 2 - double(ln 2)
__device__ double g_log_tab[65 * 3];                        // per j = 0..64: 1/F, ln F (high), ln F (low)

__device__ __forceinline__ double log64(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int m = ((hi >> 20) & 0x7ff) - 1023;
    const int mant = hi & 0xfffff;
    const int j = (mant + (1 << 13)) >> 14;                 // nearest of 64 points (0..64)
    const double y = __hiloint2double(0x3ff00000 | mant, lo);
    const double F = __hiloint2double(0x3ff00000 + (j << 14), 0);   // 1 + j/64 (j = 64: 2)
    const double f = y - F;
    const double r = f * __ldg(&g_log_tab[3 * j]);
    const double r2 = r * r;
    const double q = fma(r, fma(r, fma(r, fma(r, -1.0 / 6.0, 0.2), -0.25), 1.0 / 3.0), -0.5);
    const double p = fma(r2, q, r);
    const double md = f2d((float)m);                        // exact: |m| < 2^24
    const double head = fma(md, LN2_HI, __ldg(&g_log_tab[3 * j + 1]));
    const double tail = fma(md, LN2_LO, __ldg(&g_log_tab[3 * j + 2])) + p;
    return head + tail;
}

// The mixed path's ln T (its arguments of the Gibbs factors and FP32 forward rates):
// the same table and reduction without the low parts of ln 2 and ln F and without the
// r^6/6 term, absolute error below 5e-14 for normal x > 0 with |exponent| <= 64.
__device__ __forceinline__ double log64_mixed(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int m = ((hi >> 20) & 0x7ff) - 1023;
    const int mant = hi & 0xfffff;
    const int j = (mant + (1 << 13)) >> 14;
    const double y = __hiloint2double(0x3ff00000 | mant, lo);
    const double F = __hiloint2double(0x3ff00000 + (j << 14), 0);
    const double r = (y - F) * __ldg(&g_log_tab[3 * j]);
    const double q = fma(r, fma(r, fma(r, 0.2, -0.25), 1.0 / 3.0), -0.5);
    const double p = fma(r * r, q, r);
    return fma(f2d((float)m), LN2_HI, __ldg(&g_log_tab[3 * j + 1])) + p;
}

// FP64 instances of the bulk-type helpers (transport and chemistry of the FP64
// path): table-driven exponential and logarithm, Newton-Raphson reciprocal (the
// arguments -- viscosities, mixture sums, pressures, molar masses -- lie in the FP32
// normal range).
__device__ __forceinline__ double rcp(double x) { return rcp64(x); }
__device__ __forceinline__ double exp_(double x) { return exp64(x); }
__device__ __forceinline__ double log_(double x) { return log64(x); }

// ----------------------------------------------------------------------------- thermo

// Mixture polynomial of the specific internal energy for one NASA range:
// e(T) = e5 + T (e0 + T (e1 + T (e2 + T (e3 + T e4)))), cv(T) = de/dT.  The cv
// coefficients come in FP32 (cvf: the Newton update's derivative, and the mixed
// path's cv) and, if CV64, in FP64 (cv: the FP64 path's cv, gamma and c).
struct MixPoly {
    double e[6];
    double cv[5];
    float cvf[5];
};

// The species coefficients hold e_s = h_s - (R/W_s) T (the -R/W_s in the linear
// term); the constant term's sum starts from e5 (the Newton solve's -e_target).
template <int NS, bool CV64>
__device__ __forceinline__ void mix_poly(const MechDev &M, int r, const double (&Y)[NS], double e5, MixPoly &P) {
    double c[6] = {0, 0, 0, 0, 0, e5};
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int k = 0; k < 6; ++k) c[k] = fma(Y[s], M.ecR[r][s][k], c[k]);
    }
    // sum_s Y_s (R/W_s) [(a1 - 1) T + a2 T^2/2 + ... + a5 T^5/5 + a6] + e5
    P.e[0] = c[0];
    P.e[1] = c[1];
    P.e[2] = c[2];
    P.e[3] = c[3];
    P.e[4] = c[4];
    P.e[5] = c[5];
    // cv = c0 + 2 c1 T + 3 c2 T^2 + 4 c3 T^3 + 5 c4 T^4
    if (CV64) {
        P.cv[0] = P.e[0];
        P.cv[1] = 2.0 * c[1];
        P.cv[2] = 3.0 * c[2];
        P.cv[3] = 4.0 * c[3];
        P.cv[4] = 5.0 * c[4];
    }
    P.cvf[0] = d2f(P.e[0]);
    P.cvf[1] = 2.0f * d2f(c[1]);
    P.cvf[2] = 3.0f * d2f(c[2]);
    P.cvf[3] = 4.0f * d2f(c[3]);
    P.cvf[4] = 5.0f * d2f(c[4]);
}

// cv(T) of the mixture polynomial P in FP32 (relative error a few 1e-7).
__device__ __forceinline__ float mix_cvf(const MixPoly &P, float T) {
    return fmaf(T, fmaf(T, fmaf(T, fmaf(T, P.cvf[4], P.cvf[3]), P.cvf[2]), P.cvf[1]), P.cvf[0]);
}

__device__ __forceinline__ int nasa_range_of(const MechDev &M, double T) { return (M.two_ranges && ge_pos(T, M.Tmid)) ? 1 : 0; }

// Newton solve of e(T) = e_target, warm-started from T, with e(T) = sum_s Y_s e_s(T);
// the weights may be mass fractions (energy per unit mass)
// or partial densities (energy per unit volume, e_target = rho e: the same root, and
// the polynomial P is then density-weighted).  The residual is FP64; the derivative
// cv is the FP32 polynomial, whose relative error (a few 1e-7) only sets the
// convergence rate, not the root.  Returns false if the update did not fall below
// 1e-9 T (which leaves T within ~1e-16 T of the root, see the tolerance below) within
// maxit iterations.  On return P holds the mixture polynomial of the range containing T.
template <int NS, bool CV64>
__device__ __forceinline__ bool newton_T(const MechDev &M, const double (&Y)[NS], double e_target, double &T, int maxit,
                                         MixPoly &P) {
    int r = nasa_range_of(M, T);
    mix_poly<NS, CV64>(M, r, Y, -e_target, P);      // P.e[5] holds e5 - e_target
    // Stop once the update just applied is below 1e-9 T: the iteration contracts the
    // error by the FP32 derivative's few 1e-7 per step (plus a quadratic term), so the
    // updated T is then within ~1e-16 T of the root, and a further step (the
    // |dT| <= 1e-13 T test of the definition) would move it by less than that.
    const double tol = 1.0e-9 * fabs(T);
    for (int it = 0; it < maxit; ++it) {
        const int rn = nasa_range_of(M, T);
        if (rn != r) {
            r = rn;
            mix_poly<NS, CV64>(M, r, Y, -e_target, P);
        }
        // residual e(T) - e_target with the target folded into the constant term
        const double res = fma(T, fma(T, fma(T, fma(T, fma(T, P.e[4], P.e[3]), P.e[2]), P.e[1]), P.e[0]), P.e[5]);
        const double dT = res * f2d(__frcp_rn(mix_cvf(P, d2f(T))));
        T = T - dT;
        if (abs_le(dT, tol)) {
            if (M.two_ranges && nasa_range_of(M, T) != r) mix_poly<NS, CV64>(M, nasa_range_of(M, T), Y, -e_target, P);
            return true;
        }
    }
    return false;
}

// cv(T) of the mixture polynomial P in FP64 (needs CV64).
__device__ __forceinline__ double mix_cv(const MixPoly &P, double T) {
    return fma(T, fma(T, fma(T, fma(T, P.cv[4], P.cv[3]), P.cv[2]), P.cv[1]), P.cv[0]);
}

__device__ __forceinline__ int nasa_range(const MechDev &M, double T) { return nasa_range_of(M, T); }

// h_s/RT of species s.
__device__ __forceinline__ double h_RT(const MechDev &M, int r, int s, double T, double invT) {
    const double *c = M.ec[r][s];
    return fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[0]) + c[5] * invT;
}

// ln G_s = g_s/RT + ln(R T / p_atm), g_s/RT = h_s/RT - s_s/R, of species s in one Horner pass.
__device__ __forceinline__ double lnG(const MechDev &M, int r, int s, double T, double invT, double lnT) {
    const double *c = M.gc[r][s];
    return fma(c[6], lnT, fma(c[5], invT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[0])));
}
// ln (G_s / W_s), the same Horner pass with the constant term less ln W_s.
__device__ __forceinline__ double lnG_w(const MechDev &M, int r, int s, double T, double invT, double lnT) {
    const double *c = M.gc[r][s];
    return fma(c[6], lnT, fma(c[5], invT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), M.gc0w[r][s])));
}

// h_s/RT in the bulk type.
__device__ __forceinline__ float h_RT_bulk(const MechDev &M, int r, int s, float T, float invT) {
    const float *c = M.ecf[r][s];
    return fmaf(T, fmaf(T, fmaf(T, fmaf(T, c[4], c[3]), c[2]), c[1]), c[0]) + c[5] * invT;
}
__device__ __forceinline__ double h_RT_bulk(const MechDev &M, int r, int s, double T, double invT) {
    return h_RT(M, r, s, T, invT);
}

template <typename R>
__device__ __forceinline__ R cp_R(const MechDev &M, int r, int s, R T) {
    return fma(T, fma(T, fma(T, fma(T, mech_cpc<R>(M, r, s, 4), mech_cpc<R>(M, r, s, 3)), mech_cpc<R>(M, r, s, 2)),
                      mech_cpc<R>(M, r, s, 1)),
               mech_cpc<R>(M, r, s, 0));
}

// ----------------------------------------------------------------------------- transport

// Wilke mixture viscosity and conductivity, mixture-averaged diffusion
// coefficients Dc_s = rho D_s W_s / Wbar.  Ts = T / 300.
template <typename R, int NS>
__device__ __forceinline__ void transport(const MechDev &M, int rng, R T, R p, R rho, R Wbar, const R (&X)[NS],
                                          R &mu, R &lam, R (&Dc)[NS], R &Dmax) {
    const R lnTs = log_(T * R(1.0 / 300.0));
    R mus[NS], sq[NS], isq[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if constexpr (sizeof(R) == 8) {
            // sqrt(mu_s) and its reciprocal from one exponential pair, mu_s as its square
            exp_pair(fma(M.h_mu_exp[s], lnTs, M.hl_mu_ref[s]), sq[s], isq[s]);
            mus[s] = sq[s] * sq[s];
        } else {
            mus[s] = mech_mu_ref<R>(M, s) * exp_(mech_mu_exp<R>(M, s) * lnTs);
            sq[s] = sqrt_(mus[s]);
            isq[s] = rcp(sq[s]);
        }
    }
    R num_mu = 0, num_lam = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        R den = 0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const R a = fma(sq[i] * isq[j], mech_wc<R>(M, i, j), R(1));
            den = fma(X[j], a * a * mech_wd<R>(M, i, j), den);
        }
        const R xr = X[i] * rcp(den);
        const R cps = cp_R<R>(M, rng, i, T) * mech_RW<R>(M, i);          // cp_s, J/kg/K
        num_mu = fma(xr, mus[i], num_mu);
        num_lam = fma(xr, mus[i] * (cps + mech_eucken<R>(M, i)), num_lam);
    }
    mu = num_mu;
    lam = num_lam;
    if (NS == 1) {
        Dc[0] = 0;
        Dmax = 0;
        return;
    }
    // D_ij = D_ref,ij (T/300)^1.75 (p_atm / p)
    const R fT = exp_(R(1.75) * lnTs) * R(PATM) * rcp(p);
    R Xe[NS];
    R Wbe = 0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        Xe[j] = X[j] + R(EPS_D);
        Wbe = fma(Xe[j], mech_W<R>(M, j), Wbe);
    }
    const R rWbe = rcp(Wbe);
    const R rhoW = rho * rcp(Wbar);
    Dmax = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        R num = 0, den = 0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            if (j == s) continue;
            num = fma(Xe[j], mech_W<R>(M, j), num);
            den = fma(Xe[j], mech_invD<R>(M, s, j), den);
        }
        const R D = num * fT * rWbe * rcp(den);
        Dmax = D > Dmax ? D : Dmax;
        Dc[s] = rhoW * D * mech_W<R>(M, s);
    }
}

}  // namespace rf
