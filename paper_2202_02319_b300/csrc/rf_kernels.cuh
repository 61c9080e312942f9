// Kernels of one RHS evaluation / SSP-RK3 stage:
//   cell_state   per cell: primitives (FP64 Newton for T), transport,
//                chemistry, laser; writes the Q fields and the source-initialised RHS
//   sweep_x      x faces: LLF-split WENO3-Z inviscid + central diffusive flux,
//                divergence into the RHS (rows in chunks, carried left face)
//   sweep_walk   y or z faces, one thread per line segment walking along the axis
//   the last active sweep either accumulates, writes dU/dt, or performs the
//   Shu-Osher stage update U_out = a Un + b (U + dt L) in FP64.
#pragma once

#include "rf_device.cuh"

namespace rf {

enum SweepMode { MODE_ACCUM = 0, MODE_RHS = 1, MODE_STAGE = 2 };
enum Flags { F_NO_INVISCID = 1, F_NO_VISCOUS = 2, F_NO_CHEM = 4, F_NO_LASER = 8, F_TENO6 = 16 };

__device__ __forceinline__ int map_idx(int i, int n, int bc) {
    if (i < 0) return bc == 0 ? i + n * ((n - 1 - i) / n) : 0;
    if (i >= n) return bc == 0 ? i % n : n - 1;
    return i;
}

__device__ __forceinline__ void flag_error(const Member &m, int bits, long long cell) {
    atomicOr(m.status, bits);
    atomicCAS((unsigned long long *)m.bad_cell, (unsigned long long)(-1LL), (unsigned long long)cell);
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
    // non-negative doubles order like their bit patterns
    if (v > 0.0) atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ----------------------------------------------------------------------------- chemistry

// A finite FP64 (or FP32) value as an FP32 mantissa m with 1 <= |m| < 2 and a binary
// exponent e, value = m 2^e (m truncated to 23 fraction bits, relative error below
// 1.2e-7; zero and subnormal inputs give 2^-1023 or 2^-127 times a unit mantissa, i.e. a
// negligible value of the same sign).
struct SplitF {
    float m;
    int e;
};
__device__ __forceinline__ SplitF split64(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    SplitF r;
    r.e = (int)((hi >> 20) & 0x7ffu) - 1023;
    r.m = __uint_as_float((hi & 0x80000000u) | 0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
    return r;
}
// m 2^e in FP32 for |m| in [0.5, 64): 0 when e < -126 (a value below 2^-120), infinity
// from 2^128 on
__device__ __forceinline__ float unsplit(float m, int e) {
    const float scale = e < -126 ? 0.f : __uint_as_float((unsigned)(min(e, 128) + 127) << 23);
    return m * scale;
}
__device__ __forceinline__ SplitF split32(float x) {
    const unsigned u = __float_as_uint(x);
    SplitF r;
    r.e = (int)((u >> 23) & 0xffu) - 127;
    r.m = __uint_as_float((u & 0x807fffffu) | 0x3f800000u);
    return r;
}

// Reversible mass-action rates.  Per-species inputs sit in per-thread
// shared-memory columns (stride = block size) so the compact stoichiometry can
// index species at run time:
//   sCb = C_s in the bulk type, sP = C_s G_s and sRr = 1 / G_s (FP64),
//   G_s = exp(g_s/RT) R T / p_atm, and (rates only) sG = G_s (FP64),
// so that k_f / K_c,j * prod_s C_s^nu''_sj = k_f prod_prod (C G)_s prod_reac (1/G)_s,
// i.e. the equilibrium constant costs one FP64 exponential per species rather than
// per reaction, and the reverse rate stays in FP64.  sW accumulates
// sum_j nu_sj q_j in the bulk type.  If want_rate, sD accumulates the diagonal of
// d omega / d C and the function returns max_s |d omega_s / d rho_s|.
// Factor g of a pressure-dependent reaction j (M.ptype[j] != 0) that multiplies its
// Arrhenius k_f in both directions: [M] = sum_s eff_s C_s for a third body; for a
// fall-off P_r / (1 + P_r) F with P_r = k_0 [M] / k_inf, written 1 / (1 + exp(-ln P_r))
// from ln P_r = ln k_0 - ln k_inf + ln [M] (no quotient of rate constants that may
// underflow), Lindemann F = 1, Troe log10 F = log10 F_c / (1 + (x / (n - 0.14 x))^2),
// x = log10 P_r + c, c = -0.4 - 0.67 log10 F_c, n = 0.75 - 1.27 log10 F_c,
// F_c = (1 - alpha) exp(-T/T***) + alpha exp(-T/T*) + exp(-T**/T).  akf is the exponent
// of k_inf.  Bulk type throughout.
template <typename R, int NS>
__device__ __noinline__ R pressure_factor(const MechDev &M, int j, R akf, R T, R lnT, R invT,
                                          const R *__restrict__ sCb, int stride) {
    const int p = M.pslot[j];
    R Mc = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) Mc = fma(sizeof(R) == 8 ? (R)M.eff[p][s] : (R)M.efff[p][s], sCb[s * stride], Mc);
    if (M.ptype[j] == 1) return Mc;
    if (!(Mc > R(0))) return R(0);
    const R a0 = sizeof(R) == 8 ? (R)(M.lnA0[p] + M.b0[p] * lnT - M.Theta0[p] * invT)
                                : (R)(M.lnA0f[p] + M.b0f[p] * lnT - M.Theta0f[p] * invT);
    const R lnPr = a0 - akf + log_(Mc);
    R g = R(1) / (R(1) + exp_(-lnPr));
    if (M.ptype[j] == 3) {
        const R al = sizeof(R) == 8 ? (R)M.troe[p][0] : (R)M.troef[p][0];
        const R T3 = sizeof(R) == 8 ? (R)M.troe[p][1] : (R)M.troef[p][1];
        const R T1 = sizeof(R) == 8 ? (R)M.troe[p][2] : (R)M.troef[p][2];
        const R T2 = sizeof(R) == 8 ? (R)M.troe[p][3] : (R)M.troef[p][3];
        const R Fc = (R(1) - al) * exp_(-T / T3) + al * exp_(-T / T1) + exp_(-T2 * invT);
        const R il10 = R(0.43429448190325182765);          // 1 / ln 10
        const R lFc = log_(Fc) * il10;
        const R c = R(-0.4) - R(0.67) * lFc, n = R(0.75) - R(1.27) * lFc;
        const R x = lnPr * il10 + c;
        const R y = x / (n - R(0.14) * x);
        g *= exp_(lFc / (R(1) + y * y) * R(2.30258509299404568402));
    }
    return g;
}

// Rates of progress q_j of the reactions outside the shape classes (irreversible,
// pressure dependent, three molecules on a side), mixed path, one at a time, into sQ.
template <int NS>
__device__ __noinline__ void chemistry_q_generic(const MechDev &M, double T, double lnT, double invT,
                                                 const float *__restrict__ sCb, const double *__restrict__ sP,
                                                 const double *__restrict__ sRr, float *__restrict__ sQ, int stride) {
    const float lnTf = d2f(lnT), invTf = d2f(invT);
    for (int i = M.cls_start[4]; i < M.cls_start[5]; ++i) {
        const int j = M.cls_rx[i];
        const float a = M.lnAf[j] + M.bf[j] * lnTf - M.Thetaf[j] * invTf;
        float kf = expf(a);
        if (M.ptype[j]) kf *= pressure_factor<float, NS>(M, j, a, d2f(T), lnTf, invTf, sCb, stride);
        float cf = kf;
        for (int k = 0; k < M.n_reac[j]; ++k) cf *= sCb[M.reac[j][k] * stride];
        float q = cf;
        if (M.rev[j]) {
            const int nf = M.n_revf[j];
            double pr = 1.0;
#pragma unroll 1
            for (int k = 0; k < nf; ++k) {
                const int e = M.revf[j][k];
                pr *= e < 16 ? sP[e * stride] : sRr[(e - 16) * stride];
            }
            q = d2f(fma(-f2d(kf * M.kapf[j]), pr, f2d(cf)));
        }
        sQ[j * stride] = q;
    }
}

// Mixed path, stage with time-step rates: the diagonal of the chemistry Jacobian
// d omega_s / d C_s into sD (cleared here) and its largest magnitude, after the rates
// of progress are done: per reactant position the forward term without that factor
// (FP32); per product position the reverse term k_f G_s prod_(other products) (C G)
// prod_reac (1/G), whose factors span more than the FP32 range but only feed an FP32
// time-step estimate, as FP32 mantissas in [1, 2) with integer binary exponents (~5e-7
// relative), G from 1/G.  Pressure-dependent reactions differentiate at fixed factor.
template <int NS>
__device__ __noinline__ float chemistry_rates_mixed(const MechDev &M, double T, double lnT, double invT,
                                                    const float *__restrict__ sCb, const double *__restrict__ sP,
                                                    const double *__restrict__ sRr, float *__restrict__ sD, int stride) {
#pragma unroll
    for (int s = 0; s < NS; ++s) sD[s * stride] = 0.f;
    const float lnTf = d2f(lnT), invTf = d2f(invT);
    const bool anyp = M.npress != 0;
    for (int j = 0; j < M.nr; ++j) {
        const float a = M.lnAf[j] + M.bf[j] * lnTf - M.Thetaf[j] * invTf;
        float kf = expf(a);
        if (anyp && M.ptype[j]) kf *= pressure_factor<float, NS>(M, j, a, d2f(T), lnTf, invTf, sCb, stride);
        const int nrc = M.n_reac[j], npd = M.n_prod[j];
        if (nrc == 1) {
            const int s0 = M.reac[j][0];
            sD[s0 * stride] = fmaf((float)M.dnu_reac[j][0], kf, sD[s0 * stride]);
        } else if (nrc == 2) {
            const int s0 = M.reac[j][0], s1 = M.reac[j][1];
            const float c0 = sCb[s0 * stride], c1 = sCb[s1 * stride];
            sD[s0 * stride] = fmaf((float)M.dnu_reac[j][0], kf * c1, sD[s0 * stride]);
            sD[s1 * stride] = fmaf((float)M.dnu_reac[j][1], kf * c0, sD[s1 * stride]);
        } else if (nrc == 3) {
            const int s0 = M.reac[j][0], s1 = M.reac[j][1], s2 = M.reac[j][2];
            const float c0 = sCb[s0 * stride], c1 = sCb[s1 * stride], c2 = sCb[s2 * stride];
            sD[s0 * stride] = fmaf((float)M.dnu_reac[j][0], kf * c1 * c2, sD[s0 * stride]);
            sD[s1 * stride] = fmaf((float)M.dnu_reac[j][1], kf * c0 * c2, sD[s1 * stride]);
            sD[s2 * stride] = fmaf((float)M.dnu_reac[j][2], kf * c0 * c1, sD[s2 * stride]);
        }
        if (!M.rev[j]) continue;
        // the reactant factors are W_s / G_s: k_f prod_reac (1 / W_s) restores 1 / G_s,
        // and a product position's G_s is W_s / (W_s / G_s)
        const SplitF f0 = split32(kf * M.kapf[j]);
        float krm = f0.m;
        int kre = f0.e;
#pragma unroll 1
        for (int k2 = 0; k2 < nrc; ++k2) {
            const SplitF f = split64(sRr[M.reac[j][k2] * stride]);
            krm *= f.m;
            kre += f.e;
        }
        if (npd == 1) {
            const int s0 = M.prod[j][0];
            const SplitF ig0 = split64(sRr[s0 * stride]);
            sD[s0 * stride] = fmaf(-(float)M.dnu_prod[j][0] * M.Wf[s0], unsplit(krm * __frcp_rn(ig0.m), kre - ig0.e),
                                   sD[s0 * stride]);
        } else if (npd == 2) {
            const int s0 = M.prod[j][0], s1 = M.prod[j][1];
            const SplitF ig0 = split64(sRr[s0 * stride]), ig1 = split64(sRr[s1 * stride]);
            const SplitF p0 = split64(sP[s0 * stride]), p1 = split64(sP[s1 * stride]);
            sD[s0 * stride] = fmaf(-(float)M.dnu_prod[j][0] * M.Wf[s0],
                                   unsplit(krm * __frcp_rn(ig0.m) * p1.m, kre - ig0.e + p1.e), sD[s0 * stride]);
            sD[s1 * stride] = fmaf(-(float)M.dnu_prod[j][1] * M.Wf[s1],
                                   unsplit(krm * __frcp_rn(ig1.m) * p0.m, kre - ig1.e + p0.e), sD[s1 * stride]);
        } else {
#pragma unroll 1
            for (int k = 0; k < npd; ++k) {
                const int s = M.prod[j][k];
                const SplitF ig = split64(sRr[s * stride]);
                float pm = krm * __frcp_rn(ig.m);
                int pe = kre - ig.e;
#pragma unroll 1
                for (int k2 = 0; k2 < npd; ++k2)
                    if (k2 != k) {
                        const SplitF f = split64(sP[M.prod[j][k2] * stride]);
                        pm *= f.m;
                        pe += f.e;
                    }
                sD[s * stride] = fmaf(-(float)M.dnu_prod[j][k] * M.Wf[s], unsplit(pm, pe), sD[s * stride]);
            }
        }
    }
    float best = 0.f;
#pragma unroll
    for (int s = 0; s < NS; ++s) best = fmaxf(best, fabsf(sD[s * stride]));
    return best;
}

template <typename R, int NS>
__device__ __forceinline__ R chemistry(const MechDev &M, double T, double lnT, double invT, const double *__restrict__ sG,
                                       const R *__restrict__ sCb, const double *__restrict__ sP,
                                       const double *__restrict__ sRr, R *__restrict__ sW, R *__restrict__ sD,
                                       int stride, bool want_rate) {
    const R lnTb = narrow<R>(lnT), invTb = narrow<R>(invT);
    const bool anyp = M.npress != 0;
    for (int j = 0; j < M.nr; ++j) {
        R kf;
        if (sizeof(R) == 8) {
            const double a = M.lnA[j] + M.b[j] * lnT - M.Theta[j] * invT;
            kf = (R)exp64(a);
            if (anyp && M.ptype[j]) kf *= pressure_factor<R, NS>(M, j, (R)a, (R)T, (R)lnT, (R)invT, sCb, stride);
        } else {
            const float a = M.lnAf[j] + M.bf[j] * (float)lnTb - M.Thetaf[j] * (float)invTb;
            kf = (R)expf(a);
            if (anyp && M.ptype[j]) kf *= pressure_factor<R, NS>(M, j, (R)a, narrow<R>(T), lnTb, invTb, sCb, stride);
        }
        const int nrc = M.n_reac[j], npd = M.n_prod[j];
        R cf = kf;
        for (int k = 0; k < nrc; ++k) cf *= sCb[M.reac[j][k] * stride];
        R q = cf;
        if (M.rev[j]) {
            // k_f (cf / k_f - prod_prod (C G) prod_reac (1/G)) with the reverse term in FP64;
            // a loop (not unrolled), so that no multiplication is issued for absent factors
            const int nf = M.n_revf[j];
            auto fac = [&](int k) {
                const int e = M.revf[j][k];
                return e < 16 ? sP[e * stride] : sRr[(e - 16) * stride];
            };
            double pr = nf > 0 ? fac(0) : 1.0;
#pragma unroll 1
            for (int k = 1; k < nf; ++k) pr *= fac(k);
            q = narrow<R>(fma(-wide(kf), pr, wide(cf)));
        }
        for (int k = 0; k < M.n_net[j]; ++k) {
            const int s = M.net_sp[j][k];
            sW[s * stride] = fma((R)M.net_nu[j][k], q, sW[s * stride]);
        }
        if (want_rate) {
            // d q / d C_s at each position of the reactant / product lists (a species
            // repeated by its coefficient appears at as many positions): the forward term
            // without that reactant factor, in the bulk type ...
            // (straight-line code per reactant count, the same for every thread; products
            // in list order)
            if (nrc == 1) {
                const int s0 = M.reac[j][0];
                sD[s0 * stride] = fma((R)M.dnu_reac[j][0], kf, sD[s0 * stride]);
            } else if (nrc == 2) {
                const int s0 = M.reac[j][0], s1 = M.reac[j][1];
                const R c0 = sCb[s0 * stride], c1 = sCb[s1 * stride];
                sD[s0 * stride] = fma((R)M.dnu_reac[j][0], kf * c1, sD[s0 * stride]);
                sD[s1 * stride] = fma((R)M.dnu_reac[j][1], kf * c0, sD[s1 * stride]);
            } else if (nrc == 3) {
                const int s0 = M.reac[j][0], s1 = M.reac[j][1], s2 = M.reac[j][2];
                const R c0 = sCb[s0 * stride], c1 = sCb[s1 * stride], c2 = sCb[s2 * stride];
                sD[s0 * stride] = fma((R)M.dnu_reac[j][0], kf * c1 * c2, sD[s0 * stride]);
                sD[s1 * stride] = fma((R)M.dnu_reac[j][1], kf * c0 * c2, sD[s1 * stride]);
                sD[s2 * stride] = fma((R)M.dnu_reac[j][2], kf * c0 * c1, sD[s2 * stride]);
            }
            // ... and the reverse term k_f G_s prod_(other products) (C G) prod_reac (1/G),
            // the reactant factors shared by every product position.  FP64 path: in FP64.
            // Mixed path: the factors span more than the FP32 range but the result only
            // feeds the FP32 accumulator of a time-step estimate, so each factor is an
            // FP32 mantissa in [1, 2) with an integer binary exponent (~5e-7 relative), and
            // G comes from 1/G, so that no FP64 copy of G is kept.
            if (sizeof(R) == 4 && M.rev[j]) {
                const SplitF f0 = split32(kf);
                float krm = f0.m;
                int kre = f0.e;
#pragma unroll 1
                for (int k2 = 0; k2 < nrc; ++k2) {
                    const SplitF f = split64(sRr[M.reac[j][k2] * stride]);
                    krm *= f.m;
                    kre += f.e;
                }
                if (npd == 1) {
                    const int s0 = M.prod[j][0];
                    const SplitF ig0 = split64(sRr[s0 * stride]);      // G = 1 / (1/G)
                    sD[s0 * stride] = fma(-(R)M.dnu_prod[j][0], (R)unsplit(krm * __frcp_rn(ig0.m), kre - ig0.e),
                                          sD[s0 * stride]);
                } else if (npd == 2) {
                    const int s0 = M.prod[j][0], s1 = M.prod[j][1];
                    const SplitF ig0 = split64(sRr[s0 * stride]), ig1 = split64(sRr[s1 * stride]);
                    const SplitF p0 = split64(sP[s0 * stride]), p1 = split64(sP[s1 * stride]);
                    sD[s0 * stride] = fma(-(R)M.dnu_prod[j][0],
                                          (R)unsplit(krm * __frcp_rn(ig0.m) * p1.m, kre - ig0.e + p1.e), sD[s0 * stride]);
                    sD[s1 * stride] = fma(-(R)M.dnu_prod[j][1],
                                          (R)unsplit(krm * __frcp_rn(ig1.m) * p0.m, kre - ig1.e + p0.e), sD[s1 * stride]);
                } else {
#pragma unroll 1
                    for (int k = 0; k < npd; ++k) {
                        const int s = M.prod[j][k];
                        const SplitF ig = split64(sRr[s * stride]);
                        float pm = krm * __frcp_rn(ig.m);
                        int pe = kre - ig.e;
#pragma unroll 1
                        for (int k2 = 0; k2 < npd; ++k2)
                            if (k2 != k) {
                                const SplitF f = split64(sP[M.prod[j][k2] * stride]);
                                pm *= f.m;
                                pe += f.e;
                            }
                        sD[s * stride] = fma(-(R)M.dnu_prod[j][k], (R)unsplit(pm, pe), sD[s * stride]);
                    }
                }
            } else if (M.rev[j]) {
                double kr = wide(kf);
#pragma unroll 1
                for (int k2 = 0; k2 < nrc; ++k2) kr *= sRr[M.reac[j][k2] * stride];
#pragma unroll 1
                for (int k = 0; k < npd; ++k) {
                    const int s = M.prod[j][k];
                    double part = kr * sG[s * stride];
#pragma unroll 1
                    for (int k2 = 0; k2 < npd; ++k2)
                        if (k2 != k) part *= sP[M.prod[j][k2] * stride];
                    sD[s * stride] = fma(-(R)M.dnu_prod[j][k], narrow<R>(part), sD[s * stride]);
                }
            }
        }
    }
    R best = 0;
    if (want_rate) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const R d = fabs(sD[s * stride]);
            best = d > best ? d : best;
        }
    }
    return best;
}

// Per-species chemistry inputs of one cell (see chemistry()).
template <typename R, int NS>
__device__ __forceinline__ void chemistry_inputs(const MechDev &M, int rng, const double (&rs)[NS], double T, double invT,
                                                 double lnT, double *sG, R *sCb, double *sP, double *sRr, R *sW, R *sD,
                                                 int stride, bool rates) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double G, iG;
        if (sizeof(R) == 4) {
            // mixed path: G' = G_s / W_s from the folded constant, so C_s G_s = rho_s G'
            // takes one FP64 product and the reactant factors are W_s / G_s (the
            // reverse term carries prod_reac 1 / W_s in FP32 with k_f); C_s in FP32
            exp_pair_mixed(lnG_w(M, rng, s, T, invT, lnT), G, iG);
            sCb[s * stride] = (R)(d2f(rs[s]) * M.invWf[s]);
            sP[s * stride] = rs[s] * G;
        } else {
            const double C = rs[s] * M.invW[s];
            exp_pair(lnG(M, rng, s, T, invT, lnT), G, iG);
            sCb[s * stride] = narrow<R>(C);
            sP[s * stride] = C * G;
        }
        sRr[s * stride] = iG;
        sW[s * stride] = (R)0;
        if (rates) {
            if (sizeof(R) == 8) sG[s * stride] = G;
            sD[s * stride] = (R)0;
        }
    }
}

// ----------------------------------------------------------------------------- cell state

// Dynamic shared memory of one cell-state block of B threads: per species and thread
// C G and 1/G (FP64) and C (bulk type); then, mixed path, the rates of progress q_j per
// reaction (max(NS, nr) columns), which the rate-Jacobian diagonal of the time-step
// evaluation reuses once omega is formed; FP64 path, the per-species rate accumulator
// and, with rates, the Jacobian diagonal and G (FP64), placed last so that launches
// without rates need less.
template <typename R, int NS>
__host__ __device__ constexpr size_t cell_state_smem(int B, bool rates, int nr) {
    return sizeof(R) == 4
               ? (size_t)B * (NS * (2 * sizeof(double) + sizeof(R)) + (size_t)(nr > NS ? nr : NS) * sizeof(R))
               : (size_t)B * NS *
                     (2 * sizeof(double) + 2 * sizeof(R) + (rates ? sizeof(R) + (sizeof(R) == 8 ? sizeof(double) : 0) : 0));
}
template <typename R, int NS>
__host__ __device__ constexpr size_t cell_state_smem_max(int B, int nr) {
    return cell_state_smem<R, NS>(B, true, nr) > cell_state_smem<R, NS>(B, false, nr) ? cell_state_smem<R, NS>(B, true, nr)
                                                                                     : cell_state_smem<R, NS>(B, false, nr);
}

// Rate of progress of a reversible elementary reaction j with NRC reactant and NPD
// product molecules (mixed path): k_f in FP32, the forward term k_f prod C in FP32,
// the reverse factors prod_prod (C G) prod_reac (1/G) in FP64 (as a two-level product)
// and q = k_f (prod C - reverse factors) joined by one FP64 FMA.
template <int NRC, int NPD>
__device__ __forceinline__ float q_elementary(const MechDev &M, int j, float lnT, float invT, const float *__restrict__ sCb,
                                              const double *__restrict__ sP, const double *__restrict__ sRr, int stride) {
    const float kf = expf(M.lnAf[j] + M.bf[j] * lnT - M.Thetaf[j] * invT);
    const int r0 = M.reac[j][0] * stride, p0 = M.prod[j][0] * stride;
    float cf = kf * sCb[r0];
    double pp = sP[p0], rr = sRr[r0];
    if (NRC == 2) {
        const int r1 = M.reac[j][1] * stride;
        cf *= sCb[r1];
        rr *= sRr[r1];
    }
    if (NPD == 2) pp *= sP[M.prod[j][1] * stride];
    return d2f(fma(-f2d(kf * M.kapf[j]), pp * rr, f2d(cf)));
}

// The rates of progress of one shape class, two reactions per iteration so that their
// independent FP64 products overlap (an odd last reaction is computed twice).
template <int NRC, int NPD>
__device__ __forceinline__ void q_class(const MechDev &M, int c, float lnT, float invT, const float *__restrict__ sCb,
                                        const double *__restrict__ sP, const double *__restrict__ sRr, float *__restrict__ sQ,
                                        int stride) {
    const int i0 = M.cls_start[c], i1 = M.cls_start[c + 1];
#pragma unroll 1
    for (int i = i0; i < i1; i += 2) {
        const int ja = M.cls_rx[i], jb = M.cls_rx[i + 1 < i1 ? i + 1 : i];
        const float qa = q_elementary<NRC, NPD>(M, ja, lnT, invT, sCb, sP, sRr, stride);
        const float qb = q_elementary<NRC, NPD>(M, jb, lnT, invT, sCb, sP, sRr, stride);
        sQ[ja * stride] = qa;
        sQ[jb * stride] = qb;
    }
}

template <typename R, int NS>
__device__ __forceinline__ void cell_state_block(const MechDev &M, const Member &m, long long blk, unsigned char *smem_raw,
                                                 int newton_maxit) {
    constexpr int NV = NS + 4;
    const int B = blockDim.x;
    // sP, sRr (FP64), sCb, sW (bulk type; in the mixed path without rates sW holds q_j) |
    // rates only: sD (bulk type), FP64 path sG (FP64)
    double *sP = (double *)smem_raw;
    double *sRr = sP + NS * B;
    R *sCb = (R *)(sRr + NS * B);
    R *sW = sCb + NS * B;
    R *sD = sW + NS * B;
    double *sG = (double *)(sD + NS * B);
    __shared__ double s_laser[5];
    __shared__ R s_red[3][32];

    const int tid = threadIdx.x;
    const long long n = m.n;
    const long long cell = m.c_lo + blk * B + tid;
    const bool chem_on = !(m.flags & F_NO_CHEM) && M.nr > 0;
    const bool laser_on = m.laser_on && !(m.flags & F_NO_LASER);
    if (tid == 0 && laser_on) {
        // temporal factor at the stage time (the rest was formed on the host); the
        // exponent is bounded so that the table exponential stays in its range
        const double t = m.t_from_host ? m.t_host : m.clock[0] + m.stage_c * m.clock[1];
        const double tt = (t - m.las[5]) * m.las_k[2];
        const double a = -0.5 * tt * tt;
        s_laser[0] = a > -740.0 ? m.las_k[0] * exp64(a) : 0.0;
        s_laser[1] = m.las_k[1];
        for (int d = 0; d < 3; ++d) s_laser[2 + d] = m.las_c0[d];
    }
    __syncthreads();

    R r_ac = 0, r_df = 0, r_ch = 0;
    if (cell < m.c_hi) {
        const double *U = m.U;
        double rs[NS], Y[NS];
        double rho = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rs[s] = U[s * n + cell];
            rho += rs[s];
        }
        const double mx = U[(NS + 0) * n + cell], my = U[(NS + 1) * n + cell], mz = U[(NS + 2) * n + cell];
        const double E = U[(NS + 3) * n + cell];
        const double irho = rcp64(rho);
        // Newton on the density-weighted energy rho e(T) = sum_s rho_s e_s(T) = E - |rho u|^2 / (2 rho):
        // the same root as e(T) = e without forming the mass fractions in FP64
        // R_m rho: FP64 in the FP64 path (p, gamma, c); the mixed path forms R_m in FP32 below
        const double rho_e = fma(-0.5 * irho, fma(mx, mx, fma(my, my, mz * mz)), E);
        double T = m.T[cell];
        MixPoly P;
        const bool ok = newton_T<NS, sizeof(R) == 8>(M, rs, rho_e, T, newton_maxit, P);
        if (!ok) flag_error(m, ST_NEWTON, cell);
        // rho > 0 and 0 < T < T_MAX, compared on the bit patterns
        const bool rho_pos = (unsigned long long)(dbits(rho) - 1) < 0x7ff0000000000000ull;
        if (!rho_pos || !in_open_pos(T, T_MAX_ADMISSIBLE)) {
            if (finite64(rho) && finite64(T)) flag_error(m, ST_RANGE, cell);
            else flag_error(m, ST_NONFINITE, cell);
        }
        if (!finite64(E) || !finite64(mx) || !finite64(my) || !finite64(mz)) flag_error(m, ST_NONFINITE, cell);
        const R irhob = narrow<R>(irho);
        R ub, vb, wb;
        if constexpr (sizeof(R) == 4) {
            ub = narrow<R>(mx) * irhob;
            vb = narrow<R>(my) * irhob;
            wb = narrow<R>(mz) * irhob;
#pragma unroll
            for (int s = 0; s < NS; ++s) Y[s] = 0.0;
        } else {
            ub = mx * irho;
            vb = my * irho;
            wb = mz * irho;
#pragma unroll
            for (int s = 0; s < NS; ++s) Y[s] = rs[s] * irho;
        }
        m.T[cell] = T;

        const int rng = nasa_range(M, T);
        const double invT = rcp64(T);
        const double lnT = sizeof(R) == 4 ? log64_mixed(T) : log64(T);
        R pb, c, cpb, irmb, Wbarb;                        // P is density-weighted
        if constexpr (sizeof(R) == 4) {
            // bulk quantities of the mixed path in FP32: R_m, cv from the FP32 mixture
            // polynomial, cp, p, gamma and c, 1 / R_m and the mean molar mass
            const float Tf = d2f(T);
            float rhoRmf = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) rhoRmf = fmaf(d2f(rs[s]), M.RWf[s], rhoRmf);
            const float Rmf = rhoRmf * irhob;
            const float cvf = mix_cvf(P, Tf) * irhob;
            cpb = cvf + Rmf;
            pb = d2f(rho) * (Rmf * Tf);
            c = sqrtf(cpb * rcp(cvf) * (Rmf * Tf));
            irmb = rcp(Rmf);
            Wbarb = (float)RU * irmb;
        } else {
            double rhoRm = 0.0;
#pragma unroll
            for (int s = 0; s < NS; ++s) rhoRm = fma(rs[s], M.RW[s], rhoRm);
            const double Rm = rhoRm * irho;
            const double cv = mix_cv(P, T) * irho;
            const double cp = cv + Rm;
            pb = rho * Rm * T;
            c = sqrt_((cp / cv) * (Rm * T));
            cpb = cp;
            irmb = rcp64(Rm);
            Wbarb = RU * irmb;
        }
        R *Q = (R *)m.Q;
        Q[Q_U * n + cell] = ub;
        Q[Q_V * n + cell] = vb;
        Q[Q_W * n + cell] = wb;
        const R Tb = narrow<R>(T), invTb = narrow<R>(invT);
        Q[Q_P * n + cell] = pb;
        Q[Q_C * n + cell] = c;
        Q[Q_T * n + cell] = Tb;
        R X[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const R Ys = sizeof(R) == 4 ? narrow<R>(rs[s]) * irhob : (R)Y[s];
            X[s] = Ys * (mech_RW<R>(M, s) * irmb);
            Q[(QL<NS>::X + s) * n + cell] = X[s];
            Q[(QL<NS>::H + s) * n + cell] = h_RT_bulk(M, rng, s, Tb, invTb) * mech_RW<R>(M, s) * Tb;
        }
        // the FP64 Gibbs factors and the FP32 transport in one basic block, so that the
        // scheduler can interleave the two pipes' work
        R mu, lam, Dc[NS], Dmax;
        if (chem_on) {
            // (the mixed path clears its Jacobian diagonal itself, in the q columns)
            chemistry_inputs<R, NS>(M, rng, rs, T, invT, lnT, sG + tid, sCb + tid, sP + tid, sRr + tid, sW + tid,
                                    sD + tid, B, m.want_rates != 0 && sizeof(R) == 8);
            transport<R, NS>(M, rng, Tb, pb, narrow<R>(rho), Wbarb, X, mu, lam, Dc, Dmax);
        } else {
            transport<R, NS>(M, rng, Tb, pb, narrow<R>(rho), Wbarb, X, mu, lam, Dc, Dmax);
        }
        Q[Q_MU * n + cell] = mu;
        Q[Q_LAM * n + cell] = lam;
#pragma unroll
        for (int s = 0; s < NS; ++s) Q[(QL<NS>::DC + s) * n + cell] = Dc[s];

        R *rhs = (R *)m.rhs;
        if (chem_on && sizeof(R) == 4) {
            // mixed path: the rates of progress by shape class (straight-line code, two
            // reactions at a time), the others one by one, then omega_s = W_s sum_j nu_sj
            // q_j from the species-major lists, in registers; with time-step rates, the
            // Jacobian diagonal afterwards in the q columns
            const float *cb = (const float *)sCb + tid;
            float *sQ = (float *)sW + tid;
            const float lnTf = d2f(lnT), invTf = d2f(invT);
            q_class<1, 1>(M, 0, lnTf, invTf, cb, sP + tid, sRr + tid, sQ, B);
            q_class<1, 2>(M, 1, lnTf, invTf, cb, sP + tid, sRr + tid, sQ, B);
            q_class<2, 1>(M, 2, lnTf, invTf, cb, sP + tid, sRr + tid, sQ, B);
            q_class<2, 2>(M, 3, lnTf, invTf, cb, sP + tid, sRr + tid, sQ, B);
            if (M.cls_start[5] > M.cls_start[4])
                chemistry_q_generic<NS>(M, T, lnT, invT, cb, sP + tid, sRr + tid, sQ, B);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                float w = 0.f;
#pragma unroll 1
                for (int e = M.sp_start[s]; e < M.sp_start[s + 1]; ++e) w = fmaf((float)M.sp_nu[e], sQ[M.sp_rx[e] * B], w);
                rhs[s * n + cell] = (R)(w * M.Wf[s]);
            }
            if (m.want_rates) r_ch = (R)chemistry_rates_mixed<NS>(M, T, lnT, invT, cb, sP + tid, sRr + tid, sQ, B);
        } else if (chem_on) {
            r_ch = chemistry<R, NS>(M, T, lnT, invT, sG + tid, sCb + tid, sP + tid, sRr + tid, sW + tid, sD + tid, B,
                                    m.want_rates != 0);
#pragma unroll
            for (int s = 0; s < NS; ++s) rhs[s * n + cell] = sW[s * B + tid] * mech_W<R>(M, s);
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) rhs[s * n + cell] = (R)0;
        }
        rhs[(NS + 0) * n + cell] = (R)0;
        rhs[(NS + 1) * n + cell] = (R)0;
        rhs[(NS + 2) * n + cell] = (R)0;
        double qL = 0.0;
        if (laser_on) {
            const long long nxy = (long long)m.nx * m.ny;
            const int k = (int)(cell / nxy);
            const long long rem = cell - (long long)k * nxy;
            const int j = (int)(rem / m.nx), i = (int)(rem - (long long)j * m.nx);
            // cell indices are below 2^24, so they convert exactly through FP32; a mapped
            // grid takes the stored cell centre
            double dx, dy, dz;
            if (m.mapped) {
                dx = m.gC[cell] - m.las[1];
                dy = m.gC[m.n + cell] - m.las[2];
                dz = m.nz > 1 ? m.gC[2 * m.n + cell] - m.las[3] : 0.0;
            } else {
                dx = fma(f2d((float)i), m.h[0], s_laser[2]);
                dy = fma(f2d((float)j), m.h[1], s_laser[3]);
                dz = m.nz > 1 ? fma(f2d((float)k), m.h[2], s_laser[4]) : 0.0;
            }
            if (sizeof(R) == 8) {
                double r2 = fma(dx, dx, dy * dy);
                if (m.nz > 1) r2 = fma(dz, dz, r2);
                qL = s_laser[0] * exp64(s_laser[1] * r2);
            } else {
                // mixed path: offsets from the cell centre in FP64, their squares in FP32
                const float dxf = d2f(dx), dyf = d2f(dy), dzf = d2f(dz);
                const float r2f = fmaf(dxf, dxf, fmaf(dyf, dyf, dzf * dzf));
                qL = s_laser[0] * f2d(expf(d2f(s_laser[1]) * r2f));
            }
        }
        rhs[(NS + 3) * n + cell] = narrow<R>(qL);
        if (sizeof(R) == 4) {
#pragma unroll
            for (int v2 = 0; v2 < NV; ++v2) m.U32[v2 * n + cell] = d2f(U[v2 * n + cell]);
        }
        if (m.want_rates) {
            R ac = 0, g2 = 1;
            if (m.mapped) {
                // sum_e |u . grad xi_e| + c |grad xi_e|; the diffusive coefficient is scaled
                // by max_e |grad xi_e|^2 (the step's rule then takes unit spacing)
                const R *__restrict__ gM = (const R *)m.gM;
                const int ne[3] = {m.nx, m.ny, m.nz};
                g2 = 0;
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if (ne[e] <= 1) continue;
                    const R a0 = gM[(3 * e) * n + cell], a1 = gM[(3 * e + 1) * n + cell], a2 = gM[(3 * e + 2) * n + cell];
                    const R m2 = a0 * a0 + a1 * a1 + a2 * a2;
                    ac += fabs(a0 * ub + a1 * vb + a2 * wb) + c * sqrt(m2);
                    g2 = m2 > g2 ? m2 : g2;
                }
            } else {
                if (m.nx > 1) ac += (fabs(ub) + c) * narrow<R>(m.invh[0]);
                if (m.ny > 1) ac += (fabs(vb) + c) * narrow<R>(m.invh[1]);
                if (m.nz > 1) ac += (fabs(wb) + c) * narrow<R>(m.invh[2]);
            }
            r_ac = ac;
            if (!(m.flags & F_NO_VISCOUS)) {
                const R rhob = narrow<R>(rho);
                const R nu = mu / rhob;
                const R al = lam / (rhob * cpb);
                R d = nu > al ? nu : al;
                r_df = Dmax > d ? Dmax : d;
                if (m.mapped) r_df *= g2;
            }
        }
    }
    if (m.want_rates) {
        // block max in the bulk type (deterministic: max is exact, and so is the
        // widening to FP64), then one atomic per block
        R a = r_ac, d = r_df, ch = r_ch;
        for (int o = 16; o > 0; o >>= 1) {
            a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
            d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
            ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, o));
        }
        const int wid = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            s_red[0][wid] = a;
            s_red[1][wid] = d;
            s_red[2][wid] = ch;
        }
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < (B + 31) / 32; ++q) {
                a = fmax(a, s_red[0][q]);
                d = fmax(d, s_red[1][q]);
                ch = fmax(ch, s_red[2][q]);
            }
            atomic_max_pos(&m.rates[0], wide(a));
            atomic_max_pos(&m.rates[1], wide(d));
            atomic_max_pos(&m.rates[2], wide(ch));
        }
    }
}

template <typename R, int NS>
// mixed path: six blocks per SM in launches without rates (27.6 KB of shared memory
// per block at 9 species); the FP64 path keeps five (more would spill heavily)
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 6 : 5) cell_state_kernel(int mslot, const __grid_constant__ Member m,
                                                         int newton_maxit) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cell_state_block<R, NS>(M, m, blockIdx.x, smem_raw, newton_maxit);
}

// ----------------------------------------------------------------------------- face flux

// WENO3-Z value at i+1/2 from (f_{i-1}, f_i, f_{i+1}) = (a, b, c) with d = (1/3, 2/3),
// p = 1 and the grid-scaled eps = e2 (a^2 + b^2 + c^2) + EPS_WENO, e2 = h^2 / 3 (h the
// spacing along the sweep): of order h^2 relative to the values' squares, which keeps
// third order at smooth extrema and makes the weights independent of each variable's
// scale.  The Z weights alpha_k = d_k (1 + tau / (beta_k + eps)) are formed after
// multiplying both by (beta_0 + eps)(beta_1 + eps) / S^2, S = beta_0 + beta_1 + 2 eps:
// omega_0 = d0 b1 (b0 + t) / (d0 b1 (b0 + t) + d1 b0 (b1 + t)) with b_k = (beta_k + eps) / S,
// t = tau / S.  Every scaled quantity lies in [0, 2], so the weights cannot overflow
// even in FP32 (values up to |f| ~ 1e19 there).
// weno3z_eps takes eps itself (the characteristic-wise splitting forms it from the
// components a field is made of).
template <typename R>
__device__ __forceinline__ R weno3z_eps(R a, R b, R c, R eps) {
    const R q0 = fma(R(-0.5), a, R(1.5) * b);
    const R q1 = R(0.5) * b + R(0.5) * c;
    const R d0 = b - a, d1 = c - b;
    const R beta0 = d0 * d0, beta1 = d1 * d1;
    const R iS = rcp(beta0 + beta1 + R(2) * eps);
    const R b0 = (beta0 + eps) * iS, b1 = (beta1 + eps) * iS;
    const R t = fabs(beta1 - beta0) * iS;
    const R a0 = R(1.0 / 3.0) * b1 * (b0 + t);
    const R a1 = R(2.0 / 3.0) * b0 * (b1 + t);
    return fma(a0, q0, a1 * q1) * rcp(a0 + a1);
}

// FP32 reciprocal from the SFU (rcp.approx: about 1 ulp), for weights and
// factors of the FP32-bulk face arithmetic whose arguments are normal numbers.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_face(float x) { return rcp_approx(x); }
__device__ __forceinline__ double rcp_face(double x) { return rcp64(x); }

// The same WENO3-Z value in FP32 with the fused operations written out: with
// d0 = b - a, d1 = c - b the candidates are q0 = b + d0/2, q1 = b + d1/2, and
// omega0 q0 + omega1 q1 = q1 + omega0 (d0 - d1)/2.  S >= 2 eps and a0 + a1 >= 1/12 are
// normal, so the SFU reciprocals apply.
template <>
__device__ __forceinline__ float weno3z_eps<float>(float a, float b, float c, float eps) {
    const float d0 = b - a, d1 = c - b;
    const float beta0 = d0 * d0, beta1 = d1 * d1;
    const float iS = rcp_approx((beta0 + beta1) + 2.0f * eps);
    const float eS = eps * iS;
    const float b0 = fmaf(beta0, iS, eS), b1 = fmaf(beta1, iS, eS);
    const float t = fabsf(beta1 - beta0) * iS;
    const float a0 = (1.0f / 3.0f) * (b1 * (b0 + t));
    const float a1 = (2.0f / 3.0f) * (b0 * (b1 + t));
    const float om0 = a0 * rcp_approx(a0 + a1);
    return fmaf(om0, 0.5f * (d0 - d1), fmaf(0.5f, d1, b));
}

// The same value in FP64.  The weights are invariant under a common scale of the
// betas and eps, so S is normalised by the exact power of two 2^-E(S) (E the exponent
// of S, read from its bits): no rounding, and no division.  a0 + a1 lies in [1/12, 4],
// so the one remaining reciprocal is the Newton-Raphson rcp64.
template <>
__device__ __forceinline__ double weno3z_eps<double>(double a, double b, double c, double eps) {
    const double d0 = b - a, d1 = c - b;
    const double beta0 = d0 * d0, beta1 = d1 * d1;
    const double S = (beta0 + beta1) + 2.0 * eps;
    const double iS = __hiloint2double((2046 - ((__double2hiint(S) >> 20) & 0x7ff)) << 20, 0);
    const double eS = eps * iS;
    const double b0 = fma(beta0, iS, eS), b1 = fma(beta1, iS, eS);
    const double t = fabs(beta1 - beta0) * iS;
    const double a0 = (1.0 / 3.0) * (b1 * (b0 + t));
    const double a1 = (2.0 / 3.0) * (b0 * (b1 + t));
    const double om0 = a0 * rcp64(a0 + a1);
    return fma(om0, 0.5 * (d0 - d1), fma(0.5, d1, b));
}

// WENO3-Z with the grid-scaled eps = e2 (a^2 + b^2 + c^2) + EPS_WENO.
__device__ __forceinline__ float weno3z_e2(float a, float b, float c, float e2) {
    return weno3z_eps<float>(a, b, c, fmaf(e2, fmaf(a, a, fmaf(b, b, c * c)), (float)EPS_WENO));
}
__device__ __forceinline__ double weno3z_e2(double a, double b, double c, double e2) {
    return weno3z_eps<double>(a, b, c, fma(e2, fma(a, a, fma(b, b, c * c)), EPS_WENO));
}
template <typename R>
__device__ __forceinline__ R weno3z(R a, R b, R c, R e2) {
    return weno3z_e2(a, b, c, e2);
}

// ----------------------------------------------------------------------------- TENO6

// TENO6 value at i+1/2 from f0..f5 = f_{i-2} .. f_{i+3} (after Fu, Hu and Adams, J.
// Comput. Phys. 305 (2016)): candidate stencils S0 = {i-1, i, i+1}, S1 = {i, i+1, i+2},
// S2 = {i-2, i-1, i}, S3 = {i, i+1, i+2, i+3} with optimal weights d = (9, 6, 1, 4) / 20;
// Jiang-Shu indicators beta_k and beta_6 of the whole stencil; tau = |beta_6 - (beta_1 +
// beta_2 + 4 beta_0) / 6|; stencil k is kept where chi_k = gamma_k / sum gamma >= C_T,
// gamma_k = (1 + tau / (beta_k + eps))^6; the value is sum over kept k of d_k q_k,
// normalised by the kept d_k.
//
// Everything is written in the first differences e_m = f_{m+1} - f_m (exact for
// neighbouring values within a factor two), so that a constant is reproduced exactly
// and FP32 indicators of smooth data are not swamped by the rounding of O(f) values:
//   q_k - f_i:  (e1 + 2 e2)/6, (4 e2 - e3)/6, (5 e1 - 2 e0)/6, (9 e2 - 4 e3 + e4)/12,
//   beta_0 = 13/12 (e2 - e1)^2 + 1/4 (e1 + e2)^2,
//   beta_1 = 13/12 (e3 - e2)^2 + 1/4 (e3 - 3 e2)^2,
//   beta_2 = 13/12 (e1 - e0)^2 + 1/4 (3 e1 - e0)^2,
//   beta_3 = 1/36 (11 e2 - 7 e3 + 2 e4)^2 + 13/12 (3 e3 - 2 e2 - e4)^2 + 781/720 (e2 - 2 e3 + e4)^2,
//   beta_6 = sum_k D_k (L_k . e)^2, an exact LDL^T factorisation of the six-point form
// (the indicators are sums of squares, so they cannot round below zero).  The cut test
// chi_k >= C_T is taken without forming gamma (which overflows): with b_k = beta_k + eps,
// s_k = gamma_k / gamma_max = b_min (b_k + tau) / (b_k (b_min + tau)) lies in (0, 1] and
// chi_k >= C_T  <=>  s_k^6 >= C_T sum_m s_m^6; b and tau are scaled by one exact power of
// two first, so the products cannot overflow.
constexpr double TENO_CT = 1.0e-7;
constexpr double TENO_EPS = 1.0e-30;

__device__ __forceinline__ float pow2_scale(float x) {       // 2^-E(x) for normal x > 0
    return __uint_as_float((unsigned)(254 - ((__float_as_uint(x) >> 23) & 0xff)) << 23);
}
__device__ __forceinline__ double pow2_scale(double x) {
    return __hiloint2double((2046 - ((__double2hiint(x) >> 20) & 0x7ff)) << 20, 0);
}
__device__ __forceinline__ float rdiv(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }

template <typename R>
__device__ __forceinline__ R teno6(R f0, R f1, R f2, R f3, R f4, R f5) {
    const R e0 = f1 - f0, e1 = f2 - f1, e2 = f3 - f2, e3 = f4 - f3, e4 = f5 - f4;
    const R q0 = (e1 + R(2) * e2) * R(1.0 / 6.0);
    const R q1 = fma(R(4), e2, -e3) * R(1.0 / 6.0);
    const R q2 = fma(R(5), e1, R(-2) * e0) * R(1.0 / 6.0);
    const R q3 = (fma(R(9), e2, R(-4) * e3) + e4) * R(1.0 / 12.0);
    auto sq = [](R x) { return x * x; };
    const R b0 = fma(R(13.0 / 12.0), sq(e2 - e1), R(0.25) * sq(e1 + e2));
    const R b1 = fma(R(13.0 / 12.0), sq(e3 - e2), R(0.25) * sq(fma(R(-3), e2, e3)));
    const R b2 = fma(R(13.0 / 12.0), sq(e1 - e0), R(0.25) * sq(fma(R(3), e1, -e0)));
    const R b3 = fma(R(1.0 / 36.0), sq(fma(R(11), e2, fma(R(-7), e3, R(2) * e4))),
                     fma(R(13.0 / 12.0), sq(fma(R(3), e3, fma(R(-2), e2, -e4))),
                         R(781.0 / 720.0) * sq(fma(R(-2), e3, e2 + e4))));
    // six-point indicator: D_k (L_k . e)^2, L_k with unit leading coefficient
    const R l0 = fma(R(-3.3800293620919937), e1, fma(R(4.137755308541131), e2,
                 fma(R(-2.2318538224071762), e3, fma(R(0.4518745009732172), e4, e0))));
    const R l1 = fma(R(-1.8788632502196132), e2, fma(R(1.2398246217680282), e3, fma(R(-0.2835945203123665), e4, e1)));
    const R l2 = fma(R(-0.8641384480158466), e3, fma(R(0.22441845180562248), e4, e2));
    const R l3 = fma(R(-0.3841978250666033), e4, e3);
    const R b6 = fma(R(2.2468501984126985), sq(l0), fma(R(3.6320275079835525), sq(l1),
                 fma(R(4.2138861378223531), sq(l2), fma(R(1.0316113515772065), sq(l3), R(0.038978122273068759) * sq(e4)))));
    const R tau = fabs(b6 - (b1 + b2 + R(4) * b0) * R(1.0 / 6.0));
    const R c0 = b0 + R(TENO_EPS), c1 = b1 + R(TENO_EPS), c2 = b2 + R(TENO_EPS), c3 = b3 + R(TENO_EPS);
    const R cmin = fmin(fmin(c0, c1), fmin(c2, c3));
    const R sc = pow2_scale(fmax(fmax(fmax(c0, c1), fmax(c2, c3)), tau));
    const R ts = tau * sc, ms = cmin * sc, mt = ms + ts;
    auto ratio = [&](R c) -> R {
        if (c <= cmin) return R(1);
        const R cs = c * sc;
        const R den = cs * mt;
        return den > R(0) ? rdiv(ms * (cs + ts), den) : R(1);
    };
    auto p6 = [&](R x) { const R x2 = x * x; return sq(x2 * x); };
    const R p0 = p6(ratio(c0)), p1 = p6(ratio(c1)), p2 = p6(ratio(c2)), p3 = p6(ratio(c3));
    const R lim = R(TENO_CT) * ((p0 + p1) + (p2 + p3));
    const R w0 = p0 >= lim ? R(9.0 / 20.0) : R(0), w1 = p1 >= lim ? R(6.0 / 20.0) : R(0);
    const R w2 = p2 >= lim ? R(1.0 / 20.0) : R(0), w3 = p3 >= lim ? R(4.0 / 20.0) : R(0);
    const R num = fma(w0, q0, fma(w1, q1, fma(w2, q2, w3 * q3)));
    return f2 + rdiv(num, (w0 + w1) + (w2 + w3));
}

// Stencil of one face along DIR read from global memory for the six-point TENO6
// flux: cells o = 0..5 are f-3 .. f+2 (L = f-1 at o = 2, R = f at o = 3).
template <typename R, typename UT, int DIR>
struct GlobalStencil6 {
    const UT *__restrict__ U;
    const R *__restrict__ Q;
    long long n;
    long long id[6];
    long long tp[3], tm[3];

    __device__ __forceinline__ GlobalStencil6(const Member &m, const UT *U_, const R *Q_, const int (&cc)[3])
        : U(U_), Q(Q_), n(m.n) {
        const long long st[3] = {1, m.nx, (long long)m.nx * m.ny};
        const int nd = DIR == 0 ? m.nx : (DIR == 1 ? m.ny : m.nz);
        const long long base = (long long)cc[0] * st[0] + (long long)cc[1] * st[1] + (long long)cc[2] * st[2] -
                               (long long)cc[DIR] * st[DIR];
#pragma unroll
        for (int o = 0; o < 6; ++o) id[o] = base + (long long)map_idx(cc[DIR] + o - 3, nd, m.bc[DIR]) * st[DIR];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == DIR) {
                tp[t] = tm[t] = 0;
                continue;
            }
            const int nt = t == 0 ? m.nx : (t == 1 ? m.ny : m.nz);
            tp[t] = (long long)(map_idx(cc[t] + 1, nt, m.bc[t]) - cc[t]) * st[t];
            tm[t] = (long long)(map_idx(cc[t] - 1, nt, m.bc[t]) - cc[t]) * st[t];
        }
    }
    __device__ __forceinline__ R u(int v, int o) const { return (R)U[v * n + id[o]]; }
    __device__ __forceinline__ R q(int f, int o) const { return Q[f * n + id[o]]; }
    __device__ __forceinline__ R qt(int f, int o, int t, bool plus) const { return Q[f * n + id[o] + (plus ? tp[t] : tm[t])]; }
};

// The four-cell view (o = 0..3 as f-2 .. f+1) of a six-cell stencil, for the
// diffusive flux, which reads L and R and their tangential neighbours only.
template <class S>
struct InnerFour {
    const S &s;
    __device__ __forceinline__ auto u(int v, int o) const { return s.u(v, o + 1); }
    __device__ __forceinline__ auto q(int f, int o) const { return s.q(f, o + 1); }
    __device__ __forceinline__ auto qt(int f, int o, int t, bool plus) const { return s.qt(f, o + 1, t, plus); }
};

// Stencil of one face along DIR read from global memory.  Cells o = 0..3 are
// f-2, f-1 (L), f (R), f+1 along DIR; qt reads the tangential neighbours of L or R.
template <typename R, typename UT, int DIR>
struct GlobalStencil {
    const UT *__restrict__ U;
    const R *__restrict__ Q;
    long long n;
    long long id[4];
    long long tp[3], tm[3];        // offsets of the +1 / -1 neighbour along each tangential axis

    __device__ __forceinline__ GlobalStencil(const Member &m, const UT *U_, const R *Q_, const int (&cc)[3])
        : U(U_), Q(Q_), n(m.n) {
        const long long st[3] = {1, m.nx, (long long)m.nx * m.ny};
        const int nd = DIR == 0 ? m.nx : (DIR == 1 ? m.ny : m.nz);
        const long long base = (long long)cc[0] * st[0] + (long long)cc[1] * st[1] + (long long)cc[2] * st[2] -
                               (long long)cc[DIR] * st[DIR];
#pragma unroll
        for (int o = 0; o < 4; ++o) id[o] = base + (long long)map_idx(cc[DIR] + o - 2, nd, m.bc[DIR]) * st[DIR];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == DIR) {
                tp[t] = tm[t] = 0;
                continue;
            }
            const int nt = t == 0 ? m.nx : (t == 1 ? m.ny : m.nz);
            tp[t] = (long long)(map_idx(cc[t] + 1, nt, m.bc[t]) - cc[t]) * st[t];
            tm[t] = (long long)(map_idx(cc[t] - 1, nt, m.bc[t]) - cc[t]) * st[t];
        }
    }
    __device__ __forceinline__ R u(int v, int o) const { return (R)U[v * n + id[o]]; }
    __device__ __forceinline__ R q(int f, int o) const { return Q[f * n + id[o]]; }
    __device__ __forceinline__ R qt(int f, int o, int t, bool plus) const { return Q[f * n + id[o] + (plus ? tp[t] : tm[t])]; }
};

// Flux G = -Fhat^a + F^d at the face between cells L = f-1 and R = f along DIR, from
// the stencil accessor st (u: conserved variables, q: Q fields, qt: tangential
// neighbours of L / R).  Every sweep variant computes its faces with this code, in
// two parts: face_visc (viscous stress, heat conduction, species diffusion: the
// only part that reads T, mu, lambda, X, Dc, h and the tangential neighbours) and
// face_invisc (the LLF-split WENO3-Z flux: conserved variables, u_n, p, c), joined
// by face_join.

// Viscous part.  ACC = false: D[s] = J_s (diffusive mass flux, subtracted),
// D[NS + k] = tau_{DIR k}, D[NS + 3] = tau . u_face - q, for face_join.  ACC = true:
// the same terms applied to the flux in D directly, as face_join would.  rho_L, rho_R
// are the sums of the partial densities of L and R when have_rho, else formed here
// (in the same order).
template <typename R, int NS, int DIR, bool ACC, class S>
__device__ __forceinline__ void face_visc(const Member &m, const S &st, R (&D)[NS + 4], R rhoL = 0, R rhoR = 0,
                                          bool have_rho = false) {
    constexpr int NV = NS + 4;
    if (!ACC) {
#pragma unroll
        for (int v = 0; v < NV; ++v) D[v] = 0;
    }
    if (!(m.flags & F_NO_VISCOUS)) {
        if (!have_rho) {
            rhoL = 0;
            rhoR = 0;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                rhoL += st.u(s, 1);
                rhoR += st.u(s, 2);
            }
        }
        const R ih = (R)m.invh[DIR];
        R velL[3], velR[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            velL[q] = st.q(Q_U + q, 1);
            velR[q] = st.q(Q_U + q, 2);
        }
        const R mu = R(0.5) * (st.q(Q_MU, 1) + st.q(Q_MU, 2));
        const R lam = R(0.5) * (st.q(Q_LAM, 1) + st.q(Q_LAM, 2));
        R dn[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) dn[q] = (velR[q] - velL[q]) * ih;
        // tangential derivatives of u_DIR and u_t along t at L and R
        R dtd[3] = {0, 0, 0}, dtt[3] = {0, 0, 0};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == DIR) continue;
            const R q4 = R(0.25) * (R)m.invh[t];
            dtd[t] = ((st.qt(Q_U + DIR, 1, t, true) - st.qt(Q_U + DIR, 1, t, false)) +
                      (st.qt(Q_U + DIR, 2, t, true) - st.qt(Q_U + DIR, 2, t, false))) * q4;
            dtt[t] = ((st.qt(Q_U + t, 1, t, true) - st.qt(Q_U + t, 1, t, false)) +
                      (st.qt(Q_U + t, 2, t, true) - st.qt(Q_U + t, 2, t, false))) * q4;
        }
        R div = dn[DIR];
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t != DIR) div += dtt[t];
        R tau[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (q == DIR) tau[q] = mu * (R(2) * dn[DIR]) - R(2.0 / 3.0) * mu * div;
            else tau[q] = mu * (dtd[q] + dn[q]);
        }
        // species diffusion with correction velocity, enthalpy flux
        R jd[NS];                   // Dc_s,face dX_s / dn
        R corr = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const R dX = (st.q(QL<NS>::X + s, 2) - st.q(QL<NS>::X + s, 1)) * ih;
            const R Dcf = R(0.5) * (st.q(QL<NS>::DC + s, 1) + st.q(QL<NS>::DC + s, 2));
            jd[s] = Dcf * dX;
            corr += jd[s];
        }
        const R irL = rcp_face(rhoL), irR = rcp_face(rhoR);
        R qh = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const R Yf = R(0.5) * (st.u(s, 1) * irL + st.u(s, 2) * irR);
            const R J = fma(Yf, corr, -jd[s]);
            const R hf = R(0.5) * (st.q(QL<NS>::H + s, 1) + st.q(QL<NS>::H + s, 2));
            qh = fma(J, hf, qh);
            if (ACC) D[s] -= J;
            else D[s] = J;
        }
        const R q = fma(-lam, (st.q(Q_T, 2) - st.q(Q_T, 1)) * ih, qh);
        R work = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (ACC) D[NS + k] += tau[k];
            else D[NS + k] = tau[k];
            work = fma(tau[k], R(0.5) * (velL[k] + velR[k]), work);
        }
        if (ACC) D[NS + 3] += work - q;
        else D[NS + 3] = work - q;
    }
}

// Inviscid part: G = -(f+ reconstructed from the left + f- from the right); rho_L,
// rho_R the sums of the partial densities of L and R met on the way (0 when the
// inviscid flux is off).
template <typename R, int NS, int DIR, class S>
__device__ __forceinline__ void face_invisc(const Member &m, const S &st, R (&G)[NS + 4], R &rhoL, R &rhoR) {
    constexpr int NV = NS + 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) G[v] = 0;
    rhoL = 0;
    rhoR = 0;
    if (!(m.flags & F_NO_INVISCID)) {
        R un[4], pp[4];
        R alpha = 0;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            un[o] = st.q(Q_U + DIR, o);
            pp[o] = st.q(Q_P, o);
            const R lam = fabs(un[o]) + st.q(Q_C, o);
            alpha = lam > alpha ? lam : alpha;
        }
        // f+- = (F(U) +- alpha U) / 2 = (u_n/2 +- alpha/2) U + (p/2 or p u_n/2 for the
        // momentum along DIR and the energy)
        const R ha = R(0.5) * alpha;
        const R e2 = (R)m.weps[DIR];
        R lp[4], lm[4], hp[4], hpu[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const R h = R(0.5) * un[o];
            lp[o] = h + ha;
            lm[o] = h - ha;
            hp[o] = R(0.5) * pp[o];
            hpu[o] = hp[o] * un[o];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R fp[4], fm[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const R Uv = st.u(v, o);
                if (v < NS) {
                    if (o == 1) rhoL += Uv;
                    if (o == 2) rhoR += Uv;
                }
                fp[o] = lp[o] * Uv;
                fm[o] = lm[o] * Uv;
                if (v == NS + DIR) {
                    fp[o] += hp[o];
                    fm[o] += hp[o];
                }
                if (v == NS + 3) {
                    fp[o] += hpu[o];
                    fm[o] += hpu[o];
                }
            }
            G[v] = -(weno3z<R>(fp[0], fp[1], fp[2], e2) + weno3z<R>(fm[3], fm[2], fm[1], e2));
        }
    }
}

// Inviscid part with TENO6 on a six-cell stencil (o = 0..5, L = 2, R = 3): f+ from
// cells f-3 .. f+2, f- mirrored, alpha the largest |u_n| + c of the six cells.
template <typename R, int NS, int DIR, class S>
__device__ __forceinline__ void face_invisc_teno(const Member &m, const S &st, R (&G)[NS + 4], R &rhoL, R &rhoR) {
    constexpr int NV = NS + 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) G[v] = 0;
    rhoL = 0;
    rhoR = 0;
    if (!(m.flags & F_NO_INVISCID)) {
        R un[6], hp[6];
        R alpha = 0;
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            un[o] = st.q(Q_U + DIR, o);
            hp[o] = R(0.5) * st.q(Q_P, o);
            const R lam = fabs(un[o]) + st.q(Q_C, o);
            alpha = lam > alpha ? lam : alpha;
        }
        const R ha = R(0.5) * alpha;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R fp[6], fm[6];
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                const R Uv = st.u(v, o);
                if (v < NS) {
                    if (o == 2) rhoL += Uv;
                    if (o == 3) rhoR += Uv;
                }
                const R h = R(0.5) * un[o];
                R extra = 0;
                if (v == NS + DIR) extra = hp[o];
                if (v == NS + 3) extra = hp[o] * un[o];
                fp[o] = fma(h + ha, Uv, extra);
                fm[o] = fma(h - ha, Uv, extra);
            }
            G[v] = -(teno6<R>(fp[0], fp[1], fp[2], fp[3], fp[4], fp[5]) + teno6<R>(fm[5], fm[4], fm[3], fm[2], fm[1], fm[0]));
        }
    }
}

// Face flux with TENO6 from global memory.
template <typename R, typename UT, int NS, int DIR>
__device__ __forceinline__ void face_flux_teno(const Member &m, const UT *__restrict__ U, const R *__restrict__ Q,
                                               const int (&cc)[3], R (&G)[NS + 4]) {
    const GlobalStencil6<R, UT, DIR> st(m, U, Q, cc);
    R rhoL, rhoR;
    face_invisc_teno<R, NS, DIR>(m, st, G, rhoL, rhoR);
    const InnerFour<GlobalStencil6<R, UT, DIR>> in{st};
    face_visc<R, NS, DIR, true>(m, in, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
}

// ----------------------------------------------------------------------------- characteristic-wise splitting

// Characteristic-wise LLF splitting on Cartesian grids (Methods, Numerical method: the
// reconstruction of characteristic instead of conserved variables, the scheme's
// optional variant).  The eigensystem of dF_n/dU of the multicomponent Euler system is
// taken at the face from the arithmetic means of the two adjacent cells' Y_s, u,
// phi_s, b and H, with
//   b = gamma - 1 = rho c^2 / p - 1,  phi_s = dp/d(rho_s) = R_s T - b (e_s - |u|^2 / 2),
//   H = (E + p) / rho,  c^2 = sum_s Y_s phi_s + b (H - |u|^2)  (the face's closure).
// For a vector (r_s, m, E) with r = sum_s r_s and dp = sum_s phi_s r_s - b u . m + b E
// the left eigenvectors give
//   u -+ c:  (dp -+ c (m_n - u_n r)) / (2 c^2),  species s:  r_s - Y_s dp / c^2,
//   tangential axis t:  m_t - u_t r,
// and the right eigenvectors (columns) are (Y_s, u -+ c n, H -+ u_n c) for u -+ c,
// (e_s, u, |u|^2 - phi_s / b) for species s and (0, t, u_t) for axis t.  The split
// fluxes f+- = ((u_n +- alpha) U + p (n + u_n e_E)) / 2 project as
// ((u_n +- alpha) w_U + p (l_mn + u_n l_E)) / 2, w_U the projection of the conserved
// vector, so each field's stencil values come from three per-cell scalars (r, dp of
// U, m_n - u_n r) and one component.  WENO3-Z gives field k the eps
// (h^2 / 3) sum_j l_kj^2 sum over its three values of f_j^2 (+ EPS_WENO): the
// component-wise eps when l is the identity; TENO6 keeps its fixed eps.

template <typename R, int NS, int DIR, int K, class S>
__device__ __forceinline__ void face_invisc_char(const MechDev &M, const Member &m, const S &st, R (&G)[NS + 4],
                                                 R &rhoL, R &rhoR) {
    constexpr int NV = NS + 4;
    constexpr int OL = K / 2 - 1, OR = K / 2;
    constexpr int TA = DIR == 0 ? 1 : 0, TB = DIR == 2 ? 1 : 2;     // tangential axes, increasing
#pragma unroll
    for (int v = 0; v < NV; ++v) G[v] = 0;
    rhoL = 0;
    rhoR = 0;
    if (m.flags & F_NO_INVISCID) return;
    R un[K], pp[K], rho[K];
    R alpha = 0;
#pragma unroll
    for (int o = 0; o < K; ++o) {
        un[o] = st.q(Q_U + DIR, o);
        pp[o] = st.q(Q_P, o);
        const R lam = fabs(un[o]) + st.q(Q_C, o);
        alpha = lam > alpha ? lam : alpha;
        R r = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) r += st.u(s, o);
        rho[o] = r;
    }
    rhoL = rho[OL];
    rhoR = rho[OR];
    // face means of Y_s, u, phi_s, b, H over the two adjacent cells
    R Y[NS], phi[NS], u[3], b = 0, H = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) Y[s] = phi[s] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int o = side == 0 ? OL : OR;
        const R ir = R(1) / rho[o];
        const R co = st.q(Q_C, o), To = st.q(Q_T, o);
        const R uo[3] = {st.q(Q_U, o), st.q(Q_V, o), st.q(Q_W, o)};
        const R ke = R(0.5) * (uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2]);
        const R bo = rho[o] * co * co / pp[o] - R(1);
        b += R(0.5) * bo;
        H += R(0.5) * (st.u(NS + 3, o) + pp[o]) * ir;
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k] += R(0.5) * uo[k];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const R RT = mech_RW<R>(M, s) * To;
            const R es = st.q(QL<NS>::H + s, o) - RT;          // e_s = h_s - R_s T
            Y[s] += R(0.5) * (st.u(s, o) * ir);
            phi[s] += R(0.5) * (RT - bo * (es - ke));
        }
    }
    const R u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    R c2 = b * (H - u2);
#pragma unroll
    for (int s = 0; s < NS; ++s) c2 = fma(Y[s], phi[s], c2);
    const R c = sqrt(c2);
    const R ic2 = R(1) / c2, h2 = R(0.5) * ic2;
    const R unf = u[DIR];
    // per-cell scalars of the projection: dp of U with the face's phi, b, u, and m_n - u_n r
    R dp[K], mn[K];
#pragma unroll
    for (int o = 0; o < K; ++o) {
        R d = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) d = fma(phi[s], st.u(s, o), d);
        const R um = u[0] * st.u(NS, o) + u[1] * st.u(NS + 1, o) + u[2] * st.u(NS + 2, o);
        dp[o] = fma(b, st.u(NS + 3, o) - um, d);
        mn[o] = fma(-unf, rho[o], st.u(NS + DIR, o));
    }
    // WENO3-Z: sums of the squared component split fluxes over each side's three values
    R gp[NV], gm[NV];
    if (K == 4) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R sp = 0, sm = 0;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const R Uv = st.u(v, o);
                R extra = 0;
                if (v == NS + DIR) extra = R(0.5) * pp[o];
                if (v == NS + 3) extra = R(0.5) * pp[o] * un[o];
                const R fpv = fma(R(0.5) * (un[o] + alpha), Uv, extra);
                const R fmv = fma(R(0.5) * (un[o] - alpha), Uv, extra);
                if (o <= 2) sp = fma(fpv, fpv, sp);
                if (o >= 1) sm = fma(fmv, fmv, sm);
            }
            gp[v] = sp;
            gm[v] = sm;
        }
    }
    const R e2 = (R)m.weps[DIR];
    // reconstruction of one field from its projected U values wU[o] and face
    // coefficients lmn, lE; returns the sum of the f+ and f- reconstructions
    auto recon = [&](const R (&wU)[K], R lmn, R lE, R epsp, R epsm) -> R {
        R wp[K], wm[K];
#pragma unroll
        for (int o = 0; o < K; ++o) {
            const R extra = R(0.5) * pp[o] * fma(un[o], lE, lmn);
            wp[o] = fma(R(0.5) * (un[o] + alpha), wU[o], extra);
            wm[o] = fma(R(0.5) * (un[o] - alpha), wU[o], extra);
        }
        if (K == 6)
            return teno6<R>(wp[0], wp[1], wp[2], wp[3], wp[4], wp[5]) + teno6<R>(wm[5], wm[4], wm[3], wm[2], wm[1], wm[0]);
        return weno3z_eps<R>(wp[0], wp[1], wp[2], epsp) + weno3z_eps<R>(wm[K - 1], wm[K - 2], wm[K - 3], epsm);
    };
    // G = -F accumulates -w times each right eigenvector
    // acoustic fields u - c (sg = -1) and u + c (sg = +1)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const R sg = a == 0 ? R(-1) : R(1);
        R wU[K];
#pragma unroll
        for (int o = 0; o < K; ++o) wU[o] = fma(sg * c, mn[o], dp[o]) * h2;
        const R lmn = fma(-b, unf, sg * c) * h2, lE = b * h2;
        R ep = 0, em = 0;
        if (K == 4) {
            R sp = 0, sm = 0;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const R l = fma(-sg * c, unf, phi[s]) * h2;
                sp = fma(l * l, gp[s], sp);
                sm = fma(l * l, gm[s], sm);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const R l = (k == DIR ? fma(-b, u[k], sg * c) : -b * u[k]) * h2;
                sp = fma(l * l, gp[NS + k], sp);
                sm = fma(l * l, gm[NS + k], sm);
            }
            sp = fma(lE * lE, gp[NS + 3], sp);
            sm = fma(lE * lE, gm[NS + 3], sm);
            ep = fma(e2, sp, R(EPS_WENO));
            em = fma(e2, sm, R(EPS_WENO));
        }
        const R w = -recon(wU, lmn, lE, ep, em);
#pragma unroll
        for (int s = 0; s < NS; ++s) G[s] = fma(Y[s], w, G[s]);
#pragma unroll
        for (int k = 0; k < 3; ++k) G[NS + k] = fma(k == DIR ? u[k] + sg * c : u[k], w, G[NS + k]);
        G[NS + 3] = fma(fma(sg * unf, c, H), w, G[NS + 3]);
    }
    // species fields; their eps sums sum_q (delta_qs - Y_s phi_q / c^2)^2 g_q as
    // g_s (1 - Y_s phi_s / c^2)^2 + (Y_s / c^2)^2 (A - phi_s^2 g_s), A = sum_q phi_q^2 g_q
    const R yb = b * ic2;
    R Ap = 0, Am = 0, gvp = 0, gvm = 0;
    if (K == 4) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const R p2 = phi[q] * phi[q];
            Ap = fma(p2, gp[q], Ap);
            Am = fma(p2, gm[q], Am);
        }
        gvp = gp[NS + 3];
        gvm = gm[NS + 3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gvp = fma(u[k] * u[k], gp[NS + k], gvp);
            gvm = fma(u[k] * u[k], gm[NS + k], gvm);
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const R yc = Y[s] * ic2;
        R wU[K];
#pragma unroll
        for (int o = 0; o < K; ++o) wU[o] = fma(-yc, dp[o], st.u(s, o));
        const R lmn = Y[s] * yb * unf, lE = -Y[s] * yb;
        R ep = 0, em = 0;
        if (K == 4) {
            const R l = fma(-yc, phi[s], R(1)), ly = Y[s] * yb, p2 = phi[s] * phi[s];
            const R rp = fmax(fma(-p2, gp[s], Ap), R(0)), rm = fmax(fma(-p2, gm[s], Am), R(0));
            const R sp = fma(l * l, gp[s], fma(yc * yc, rp, ly * ly * gvp));
            const R sm = fma(l * l, gm[s], fma(yc * yc, rm, ly * ly * gvm));
            ep = fma(e2, sp, R(EPS_WENO));
            em = fma(e2, sm, R(EPS_WENO));
        }
        const R w = -recon(wU, lmn, lE, ep, em);
        G[s] += w;
#pragma unroll
        for (int k = 0; k < 3; ++k) G[NS + k] = fma(u[k], w, G[NS + k]);
        G[NS + 3] = fma(u2 - phi[s] / b, w, G[NS + 3]);
    }
    // tangential fields
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int t = j == 0 ? TA : TB;
        R wU[K];
#pragma unroll
        for (int o = 0; o < K; ++o) wU[o] = fma(-u[t], rho[o], st.u(NS + t, o));
        R ep = 0, em = 0;
        if (K == 4) {
            R sp = gp[NS + t], sm = gm[NS + t], rp = 0, rm = 0;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                rp += gp[s];
                rm += gm[s];
            }
            sp = fma(u[t] * u[t], rp, sp);
            sm = fma(u[t] * u[t], rm, sm);
            ep = fma(e2, sp, R(EPS_WENO));
            em = fma(e2, sm, R(EPS_WENO));
        }
        const R w = -recon(wU, R(0), R(0), ep, em);
        G[NS + t] += w;
        G[NS + 3] = fma(u[t], w, G[NS + 3]);
    }
}

// Face flux with characteristic-wise splitting from global memory (TENO: TENO6 on a
// six-cell stencil, else WENO3-Z); the viscous part as in the component-wise scheme.
template <typename R, typename UT, int NS, int DIR, bool TENO>
__device__ __forceinline__ void face_flux_char(const MechDev &M, const Member &m, const UT *__restrict__ U,
                                               const R *__restrict__ Q, const int (&cc)[3], R (&G)[NS + 4]) {
    R rhoL, rhoR;
    if (TENO) {
        const GlobalStencil6<R, UT, DIR> st(m, U, Q, cc);
        face_invisc_char<R, NS, DIR, 6>(M, m, st, G, rhoL, rhoR);
        const InnerFour<GlobalStencil6<R, UT, DIR>> in{st};
        face_visc<R, NS, DIR, true>(m, in, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
    } else {
        const GlobalStencil<R, UT, DIR> st(m, U, Q, cc);
        face_invisc_char<R, NS, DIR, 4>(M, m, st, G, rhoL, rhoR);
        face_visc<R, NS, DIR, true>(m, st, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
    }
}

template <typename R, int NS>
__device__ __forceinline__ void face_join(const Member &m, const R (&D)[NS + 4], R (&G)[NS + 4]) {
    if (m.flags & F_NO_VISCOUS) return;
#pragma unroll
    for (int s = 0; s < NS; ++s) G[s] -= D[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) G[NS + k] += D[NS + k];
    G[NS + 3] += D[NS + 3];
}

template <typename R, int NS, int DIR, class S>
__device__ __forceinline__ void face_flux_core(const Member &m, const S &st, R (&G)[NS + 4]) {
    R rhoL, rhoR;
    face_invisc<R, NS, DIR>(m, st, G, rhoL, rhoR);
    face_visc<R, NS, DIR, true>(m, st, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
}

// Face flux from global memory; `cc` holds the cell's coordinates (i, j, k) with
// cc[DIR] = f.
template <typename R, typename UT, int NS, int DIR>
__device__ __forceinline__ void face_flux(const Member &m, const UT *__restrict__ U, const R *__restrict__ Q, const int (&cc)[3],
                                          R (&G)[NS + 4]) {
    const GlobalStencil<R, UT, DIR> st(m, U, Q, cc);
    face_flux_core<R, NS, DIR>(m, st, G);
}

// ----------------------------------------------------------------------------- mapped grids

// Mapped (curvilinear) grids (Methods, Numerical method: the equations mapped onto a
// uniform computational grid, U~ = U / J, F~ = (xi_x F + xi_y G + xi_z H) / J, the
// Cartesian scheme applied to the mapped fluxes).  The metric of a face is its area
// vector S (from its corners; the six of a cell sum to zero), frozen over the face's
// stencil: contravariant velocity theta = S . u, LLF speed max |theta| + c |S|,
// f+- = (theta U + p (0, S, theta) +- alpha U) / 2 reconstructed as on a Cartesian grid,
// the WENO3-Z eps with h = (V_L + V_R) / (2 |S|).  A uniform flow therefore gives every
// face exactly S . F and stays uniform.  Diffusive fluxes take physical gradients
// sum_e (d / d xi_e) grad xi_e with the mean of the two cells' metrics, dotted with S.
// Cells divide the flux difference by their volume.

// Index of face f (between cells f-1 and f along DIR) of the line through cc.
template <int DIR>
__device__ __forceinline__ long long face_index(const Member &m, const int (&cc)[3]) {
    if (DIR == 0) return (long long)cc[0] + (long long)(m.nx + 1) * (cc[1] + (long long)m.ny * cc[2]);
    if (DIR == 1) return (long long)cc[0] + (long long)m.nx * (cc[1] + (long long)(m.ny + 1) * cc[2]);
    return (long long)cc[0] + (long long)m.nx * (cc[1] + (long long)m.ny * cc[2]);
}
template <int DIR>
__device__ __forceinline__ long long face_count(const Member &m) {
    return DIR == 0 ? (long long)(m.nx + 1) * m.ny * m.nz
                    : (DIR == 1 ? (long long)m.nx * (m.ny + 1) * m.nz : (long long)m.nx * m.ny * (m.nz + 1));
}

// Inviscid part through a mapped face (four-cell stencil, WENO3-Z).
template <typename R, int NS, int DIR, class ST>
__device__ __forceinline__ void face_invisc_mapped(const Member &m, const ST &st, const R (&S)[3], R e2, R (&G)[NS + 4],
                                                   R &rhoL, R &rhoR) {
    constexpr int NV = NS + 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) G[v] = 0;
    rhoL = 0;
    rhoR = 0;
    if (m.flags & F_NO_INVISCID) return;
    const R Sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    R th[4], hp[4];
    R alpha = 0;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        th[o] = S[0] * st.q(Q_U, o) + S[1] * st.q(Q_U + 1, o) + S[2] * st.q(Q_U + 2, o);
        hp[o] = R(0.5) * st.q(Q_P, o);
        const R lam = fabs(th[o]) + st.q(Q_C, o) * Sm;
        alpha = lam > alpha ? lam : alpha;
    }
    const R ha = R(0.5) * alpha;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        R fp[4], fm[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const R Uv = st.u(v, o);
            if (v < NS) {
                if (o == 1) rhoL += Uv;
                if (o == 2) rhoR += Uv;
            }
            R extra = 0;
            if (v >= NS && v < NS + 3) extra = hp[o] * S[v - NS];
            if (v == NS + 3) extra = hp[o] * th[o];
            const R h = R(0.5) * th[o];
            fp[o] = fma(h + ha, Uv, extra);
            fm[o] = fma(h - ha, Uv, extra);
        }
        G[v] = -(weno3z<R>(fp[0], fp[1], fp[2], e2) + weno3z<R>(fm[3], fm[2], fm[1], e2));
    }
}

// Inviscid part through a mapped face with TENO6 (six-cell stencil, L = 2, R = 3).
template <typename R, int NS, int DIR, class ST>
__device__ __forceinline__ void face_invisc_teno_mapped(const Member &m, const ST &st, const R (&S)[3], R (&G)[NS + 4],
                                                        R &rhoL, R &rhoR) {
    constexpr int NV = NS + 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) G[v] = 0;
    rhoL = 0;
    rhoR = 0;
    if (m.flags & F_NO_INVISCID) return;
    const R Sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    R th[6], hp[6];
    R alpha = 0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        th[o] = S[0] * st.q(Q_U, o) + S[1] * st.q(Q_U + 1, o) + S[2] * st.q(Q_U + 2, o);
        hp[o] = R(0.5) * st.q(Q_P, o);
        const R lam = fabs(th[o]) + st.q(Q_C, o) * Sm;
        alpha = lam > alpha ? lam : alpha;
    }
    const R ha = R(0.5) * alpha;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        R fp[6], fm[6];
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const R Uv = st.u(v, o);
            if (v < NS) {
                if (o == 2) rhoL += Uv;
                if (o == 3) rhoR += Uv;
            }
            R extra = 0;
            if (v >= NS && v < NS + 3) extra = hp[o] * S[v - NS];
            if (v == NS + 3) extra = hp[o] * th[o];
            const R h = R(0.5) * th[o];
            fp[o] = fma(h + ha, Uv, extra);
            fm[o] = fma(h - ha, Uv, extra);
        }
        G[v] = -(teno6<R>(fp[0], fp[1], fp[2], fp[3], fp[4], fp[5]) + teno6<R>(fm[5], fm[4], fm[3], fm[2], fm[1], fm[0]));
    }
}

// Viscous part through a mapped face, added to G (the four-cell view: L = 1, R = 2);
// Mf the face metric (d xi_e / d x_k at 3 e + k).
template <typename R, int NS, int DIR, class ST>
__device__ __forceinline__ void face_visc_mapped(const Member &m, const ST &st, const R (&S)[3], const R (&Mf)[9],
                                                 R (&G)[NS + 4], R rhoL, R rhoR, bool have_rho) {
    if (m.flags & F_NO_VISCOUS) return;
    if (!have_rho) {
        rhoL = 0;
        rhoR = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rhoL += st.u(s, 1);
            rhoR += st.u(s, 2);
        }
    }
    // d f / d xi_e at the face: two-point along DIR, mean of the two cells' central
    // differences along the other axes; physical gradient through Mf
    auto dxi = [&](int f, int e) -> R {
        if (e == DIR) return st.q(f, 2) - st.q(f, 1);
        return R(0.25) * ((st.qt(f, 1, e, true) - st.qt(f, 1, e, false)) + (st.qt(f, 2, e, true) - st.qt(f, 2, e, false)));
    };
    auto grad = [&](int f, R (&g)[3]) {
        const R d0 = dxi(f, 0), d1 = dxi(f, 1), d2 = dxi(f, 2);
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k] = d0 * Mf[k] + d1 * Mf[3 + k] + d2 * Mf[6 + k];
    };
    const R mu = R(0.5) * (st.q(Q_MU, 1) + st.q(Q_MU, 2));
    const R lam = R(0.5) * (st.q(Q_LAM, 1) + st.q(Q_LAM, 2));
    R gu[3][3];                                  // gu[l][k] = d u_l / d x_k
#pragma unroll
    for (int l = 0; l < 3; ++l) grad(Q_U + l, gu[l]);
    const R div = gu[0][0] + gu[1][1] + gu[2][2];
    R uf[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) uf[l] = R(0.5) * (st.q(Q_U + l, 1) + st.q(Q_U + l, 2));
    // tau . S (momentum) and (tau . u) . S (work)
    R tS[3], work = 0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        R a = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R t = mu * (gu[l][k] + gu[k][l]);
            if (k == l) t -= R(2.0 / 3.0) * mu * div;
            a = fma(S[k], t, a);
        }
        tS[l] = a;
        work = fma(a, uf[l], work);
    }
    // species diffusion: J_s = -Dc_s grad X_s + Y_s sum_k Dc_k grad X_k; first pass the sum
    R corr[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        R g[3];
        grad(QL<NS>::X + s, g);
        const R Dcf = R(0.5) * (st.q(QL<NS>::DC + s, 1) + st.q(QL<NS>::DC + s, 2));
#pragma unroll
        for (int k = 0; k < 3; ++k) corr[k] = fma(Dcf, g[k], corr[k]);
    }
    const R corrS = corr[0] * S[0] + corr[1] * S[1] + corr[2] * S[2];
    const R irL = rcp_face(rhoL), irR = rcp_face(rhoR);
    R qhS = 0;                                   // sum_s (J_s . S) h_s
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        R g[3];
        grad(QL<NS>::X + s, g);
        const R Dcf = R(0.5) * (st.q(QL<NS>::DC + s, 1) + st.q(QL<NS>::DC + s, 2));
        const R Yf = R(0.5) * (st.u(s, 1) * irL + st.u(s, 2) * irR);
        const R JS = fma(Yf, corrS, -Dcf * (g[0] * S[0] + g[1] * S[1] + g[2] * S[2]));
        const R hf = R(0.5) * (st.q(QL<NS>::H + s, 1) + st.q(QL<NS>::H + s, 2));
        qhS = fma(JS, hf, qhS);
        G[s] -= JS;
    }
    R gT[3];
    grad(Q_T, gT);
    const R qS = fma(-lam, gT[0] * S[0] + gT[1] * S[1] + gT[2] * S[2], qhS);
#pragma unroll
    for (int l = 0; l < 3; ++l) G[NS + l] += tS[l];
    G[NS + 3] += work - qS;
}

// Face flux through a mapped face from global memory (cc[DIR] = f).
template <typename R, typename UT, int NS, int DIR, int SCHEME>
__device__ __forceinline__ void face_flux_mapped(const Member &m, const UT *__restrict__ U, const R *__restrict__ Q,
                                                 const int (&cc)[3], R (&G)[NS + 4]) {
    const long long fi = face_index<DIR>(m, cc), nf = face_count<DIR>(m);
    const R *__restrict__ gS = (const R *)m.gS[DIR];
    const R S[3] = {gS[fi], gS[nf + fi], gS[2 * nf + fi]};
    const R *__restrict__ gM = (const R *)m.gM;
    const double *__restrict__ gV = m.gV;
    R rhoL, rhoR;
    long long iL, iR;
    if (SCHEME == 1) {
        const GlobalStencil6<R, UT, DIR> st(m, U, Q, cc);
        face_invisc_teno_mapped<R, NS, DIR>(m, st, S, G, rhoL, rhoR);
        iL = st.id[2];
        iR = st.id[3];
        R Mf[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Mf[q] = R(0.5) * (gM[q * m.n + iL] + gM[q * m.n + iR]);
        const InnerFour<GlobalStencil6<R, UT, DIR>> in{st};
        face_visc_mapped<R, NS, DIR>(m, in, S, Mf, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
    } else {
        const GlobalStencil<R, UT, DIR> st(m, U, Q, cc);
        iL = st.id[1];
        iR = st.id[2];
        const R Sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        const R hf = narrow<R>(0.5 * (gV[iL] + gV[iR])) / Sm;
        face_invisc_mapped<R, NS, DIR>(m, st, S, hf * hf * R(1.0 / 3.0), G, rhoL, rhoR);
        R Mf[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Mf[q] = R(0.5) * (gM[q * m.n + iL] + gM[q * m.n + iR]);
        face_visc_mapped<R, NS, DIR>(m, st, S, Mf, G, rhoL, rhoR, !(m.flags & F_NO_INVISCID));
    }
}

// Stage value of one conserved variable, U_out = a U^n + b (U^(k) + dt L), in FP64.
// FP64 bulk: as written.  FP32 bulk: L carries FP32 precision, so the increment
// b dt L is formed in FP32 (and widened exactly) and joined to a U^n + b U^(k) by two
// FP64 FMAs; the first stage (a = 0, b = 1) is U^(k) + dt L without reading U^n.
struct StageK {
    double a, b, dt;
    float dtf, bdtf;
    bool euler;
};
__device__ __forceinline__ StageK stage_k(const Member &m, double dt) {
    StageK k;
    k.a = m.stage_a;
    k.b = m.stage_b;
    k.dt = dt;
    k.euler = m.stage_a == 0.0 && m.stage_b == 1.0;
    k.dtf = d2f(dt);
    k.bdtf = d2f(m.stage_b * dt);
    return k;
}
__device__ __forceinline__ double stage_value(const StageK &k, double L, double uk, double un) {
    return k.euler ? fma(k.dt, L, uk) : fma(k.a, un, k.b * fma(k.dt, L, uk));
}
__device__ __forceinline__ double stage_value(const StageK &k, float L, double uk, double un) {
    return k.euler ? uk + f2d(k.dtf * L) : fma(k.a, un, fma(k.b, uk, f2d(k.bdtf * L)));
}

template <typename R, int NS, int MODE>
__device__ __forceinline__ void cell_update(const Member &m, long long cell, const R (&dG)[NS + 4], R ih) {
    constexpr int NV = NS + 4;
    const long long n = m.n;
    R *__restrict__ rhs = (R *)m.rhs;
    if (MODE == MODE_ACCUM) {
#pragma unroll
        for (int v = 0; v < NV; ++v) rhs[v * n + cell] = fma(dG[v], ih, rhs[v * n + cell]);
    } else if (MODE == MODE_RHS) {
#pragma unroll
        for (int v = 0; v < NV; ++v) m.dUdt[v * n + cell] = wide(fma(dG[v], ih, rhs[v * n + cell]));
    } else {
        const StageK k = stage_k(m, m.clock[1]);
        const double *__restrict__ Uk = m.U;
        const double *__restrict__ Un = m.Un;
        double *__restrict__ Uo = m.Uout;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const R L = fma(dG[v], ih, rhs[v * n + cell]);
            Uo[v * n + cell] = stage_value(k, L, Uk[v * n + cell], k.euler ? 0.0 : Un[v * n + cell]);
        }
    }
}

// x sweep: each block row group processes its rows in chunks of W faces; face
// f = c W + lx goes to slot lx+1, slot 0 carries the previous chunk's last face.
template <typename R, typename UT, int NS, int MODE, int SCHEME = 0, int GEOM = 0>
__device__ __forceinline__ void sweep_x_block(const MechDev &M, const Member &m, int blk, int W, int rpb,
                                              unsigned char *smem_raw) {
    constexpr int NV = NS + 4;
    R *sG = (R *)smem_raw;                       // [NV][rpb][W + 1]
    R *s0 = sG + (size_t)NV * rpb * (W + 1);     // [NV][rpb]: face 0 of each row (periodic wrap)
    const int tid = threadIdx.x;
    const int r = tid / W, lx = tid - r * W;
    const int nrows = m.ny * m.nz;
    const int row = blk * rpb + r;
    const bool active = r < rpb && row < nrows;
    const int j = active ? row % m.ny : 0, k = active ? row / m.ny : 0;
    const UT *U = (sizeof(UT) == 4) ? (const UT *)m.U32 : (const UT *)m.U;
    const R *Q = (const R *)m.Q;
    const int nx = m.nx;
    const bool periodic = m.bc[0] == 0;
    const R ih = (R)m.invh[0];
    const int nchunks = (nx + 1 + W - 1) / W;
    auto slot = [&](int v, int s) -> R & { return sG[((size_t)v * rpb + r) * (W + 1) + s]; };
    for (int c = 0; c < nchunks; ++c) {
        const int f = c * W + lx;
        // a mapped periodic row computes face nx too (its area vector is its own)
        if (active && (f < nx || (f == nx && (!periodic || GEOM)))) {
            R G[NV];
            const int cc[3] = {f, j, k};
            if (GEOM) face_flux_mapped<R, UT, NS, 0, SCHEME>(m, U, Q, cc, G);
            else if (SCHEME >= 2) face_flux_char<R, UT, NS, 0, SCHEME == 3>(M, m, U, Q, cc, G);
            else if (SCHEME == 1) face_flux_teno<R, UT, NS, 0>(m, U, Q, cc, G);
            else face_flux<R, UT, NS, 0>(m, U, Q, cc, G);
#pragma unroll
            for (int v = 0; v < NV; ++v) slot(v, lx + 1) = G[v];
            if (f == 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) s0[v * rpb + r] = G[v];
            }
        }
        __syncthreads();
        if (active && f >= 1 && f <= nx) {
            R dG[NV];
            const bool wrap = (f == nx && periodic && !GEOM);
#pragma unroll
            for (int v = 0; v < NV; ++v) dG[v] = (wrap ? s0[v * rpb + r] : slot(v, lx + 1)) - slot(v, lx);
            const long long cell = ((long long)k * m.ny + j) * nx + (f - 1);
            cell_update<R, NS, MODE>(m, cell, dG, GEOM ? ((const R *)m.giV)[cell] : ih);
        }
        __syncthreads();
        if (active) {
            for (int v = lx; v < NV; v += W) slot(v, 0) = slot(v, W);
        }
        __syncthreads();
    }
}

// SCHEME 0: WENO3-Z, 1: TENO6, 2 / 3: WENO3-Z / TENO6 characteristic-wise (Cartesian
// only); GEOM 1: mapped grid
template <typename R, typename UT, int NS, int MODE, int SCHEME = 0, int GEOM = 0>
__global__ void __launch_bounds__(256) sweep_x_kernel(int mslot, const __grid_constant__ Member m,
                                                      int W, int rpb) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep_x_block<R, UT, NS, MODE, SCHEME, GEOM>(M, m, blockIdx.x, W, rpb, smem_raw);
}

// FP32 global-memory x sweeps with a register cap: blocks of at most 128 threads, MINB
// of them per SM (the characteristic-wise, TENO6 and mapped sweeps, whose many live
// values otherwise leave 8-16 warps per SM to cover their global loads).
template <typename UT, int NS, int MODE, int SCHEME, int GEOM, int MINB>
__global__ void __launch_bounds__(128, MINB) sweep_x_capped_kernel(int mslot, const __grid_constant__ Member m, int W,
                                                                   int rpb) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep_x_block<float, UT, NS, MODE, SCHEME, GEOM>(M, m, blockIdx.x, W, rpb, smem_raw);
}

// y / z sweep: thread = one line (x fastest), segment of `seg` cells along DIR.
template <typename R, typename UT, int NS, int DIR, int MODE, int SCHEME = 0, int GEOM = 0>
__device__ __forceinline__ void sweep_walk_block(const MechDev &M, const Member &m, long long lblk, int sblk, int seg) {
    constexpr int NV = NS + 4;
    const long long line = lblk * blockDim.x + threadIdx.x;
    const int nd = DIR == 1 ? m.ny : m.nz;
    const int no = DIR == 1 ? m.nz : m.ny;
    if (line >= (long long)m.nx * no) return;
    const int x = (int)(line % m.nx), o = (int)(line / m.nx);
    const int c0 = sblk * seg;
    if (c0 >= nd) return;
    const int c1 = min(c0 + seg, nd);
    const UT *U = (sizeof(UT) == 4) ? (const UT *)m.U32 : (const UT *)m.U;
    const R *Q = (const R *)m.Q;
    const R ih = (R)m.invh[DIR];
    int cc[3];
    cc[0] = x;
    if (DIR == 1) cc[2] = o;
    else cc[1] = o;
    R Gp[NV], Gn[NV];
    const long long sd = DIR == 1 ? (long long)m.nx : (long long)m.nx * m.ny;
    const long long cbase = DIR == 1 ? ((long long)o * m.ny) * m.nx + x : (long long)o * m.nx + x;
    // one call site of face_flux, so every face is computed by the same code
    // whichever segment computes it (bitwise independence of the segmentation)
    for (int c = c0 - 1; c < c1; ++c) {
        cc[DIR] = c + 1;
        if (GEOM) face_flux_mapped<R, UT, NS, DIR, SCHEME>(m, U, Q, cc, Gn);
        else if (SCHEME >= 2) face_flux_char<R, UT, NS, DIR, SCHEME == 3>(M, m, U, Q, cc, Gn);
        else if (SCHEME == 1) face_flux_teno<R, UT, NS, DIR>(m, U, Q, cc, Gn);
        else face_flux<R, UT, NS, DIR>(m, U, Q, cc, Gn);
        if (c >= c0) {
            R dG[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) dG[v] = Gn[v] - Gp[v];
            const long long cell = cbase + (long long)c * sd;
            cell_update<R, NS, MODE>(m, cell, dG, GEOM ? ((const R *)m.giV)[cell] : ih);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Gp[v] = Gn[v];
    }
}

template <typename R, typename UT, int NS, int DIR, int MODE, int SCHEME = 0, int GEOM = 0>
__global__ void __launch_bounds__(128) sweep_walk_kernel(int mslot, const __grid_constant__ Member m,
                                                         int seg) {
    const MechDev &M = c_mech[mslot];
    sweep_walk_block<R, UT, NS, DIR, MODE, SCHEME, GEOM>(M, m, blockIdx.x, blockIdx.y, seg);
}

// FP32 global-memory y / z sweeps with a register cap (MINB blocks of 128 threads per SM):
// the characteristic-wise sweeps (latency-bound on their global loads at 221-244
// registers) and the TENO6 and mapped ones.
template <typename UT, int NS, int DIR, int MODE, int SCHEME, int GEOM, int MINB>
__global__ void __launch_bounds__(128, MINB) sweep_walk_capped_kernel(int mslot, const __grid_constant__ Member m,
                                                                      int seg) {
    const MechDev &M = c_mech[mslot];
    sweep_walk_block<float, UT, NS, DIR, MODE, SCHEME, GEOM>(M, m, blockIdx.x, blockIdx.y, seg);
}

// ----------------------------------------------------------------------------- staged y / z sweep (FP32 bulk)

// Asynchronous global -> shared copies (cp.async, completion tracked per thread by
// commit groups).  Global sources must be 4- or 16-byte aligned as the size says.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Tile of the staged walk: 32 lines along x (one warp) times 4 lines along the
// other axis o (o = z for the y sweep, y for the z sweep), 128 threads, one line
// per thread.  Shared memory holds rings of planes (cells of the tile at one
// position along DIR):
//   ring I (depth 5): the NS + 4 conserved variables (FP32 copy), u_DIR, p, c of
//                     every line: the four stencil planes of a face plus one ahead;
//   ring V (depth 3): the Q fields T, mu, lambda, X_s, Dc_s, h_s: planes L, R, ahead;
//   slab   (depth 3): u, v, w on the tile plus a one-cell halo in x and o, for the
//                     tangential derivatives of the viscous flux.
template <int NS>
struct WalkTile {
    static constexpr int TX = 32, TY = 4, NL = TX * TY;
    static constexpr int NV = NS + 4, NI = NV + 3, NVV = 3 + 3 * NS;
    static constexpr int SX = TX + 2, SY = TY + 2, NSL = SX * SY;
    static constexpr int DI = 5, DV = 2;
    static constexpr int I_FLOATS = DI * NI * NL, V_FLOATS = DV * NVV * NL, S_FLOATS = DV * 3 * NSL;
    static constexpr size_t SMEM = sizeof(float) * (size_t)(I_FLOATS + V_FLOATS + S_FLOATS);
};

template <int NS, int DIR>
struct WalkStencil {
    using W = WalkTile<NS>;
    const float *I[4];      // ring I slots of cells f-2 .. f+1: [NI][NL]
    const float *V[2];      // ring V slots of L, R: [NVV][NL]
    const float *S[2];      // slab slots of L, R: [3][NSL]
    int l, sl;              // the thread's line in the ring and in the slab
    __device__ __forceinline__ float u(int v, int o) const { return I[o][v * W::NL + l]; }
    __device__ __forceinline__ float q(int f, int o) const {
        if (f == Q_U + DIR) return I[o][(W::NV + 0) * W::NL + l];
        if (f == Q_P) return I[o][(W::NV + 1) * W::NL + l];
        if (f == Q_C) return I[o][(W::NV + 2) * W::NL + l];
        if (f < 3) return S[o - 1][f * W::NSL + sl];
        return V[o - 1][(f - Q_T) * W::NL + l];
    }
    __device__ __forceinline__ float qt(int f, int o, int t, bool plus) const {
        const int d = t == 0 ? 1 : W::SX;
        return S[o - 1][f * W::NSL + sl + (plus ? d : -d)];
    }
};

// One tile line group walking faces c0 .. c1 of its segment [c0, c1) along DIR:
// face f needs planes f-2 .. f+1 (ring I) and f-1, f (ring V, slab).  Per face: wait
// for its planes; start plane f+2 of ring I (into the slot of plane f-3); the
// viscous part (the only reader of ring V and the slab); barrier; start plane f+1
// of ring V and the slab (into the slots of plane f-1); the inviscid part and the
// update of cell f-1.  Two V slots instead of three keep a block at 74.8 KB, three
// per SM.
template <int NS, int DIR, int MODE>
__device__ __forceinline__ void sweep_walk_staged_block(const MechDev &M, const Member &m, int tile, int sblk, int seg,
                                                        float *smem) {
    using W = WalkTile<NS>;
    constexpr int NV = W::NV, NL = W::NL;
    const int nd = DIR == 1 ? m.ny : m.nz;
    const int no = DIR == 1 ? m.nz : m.ny;
    const int bco = DIR == 1 ? m.bc[2] : m.bc[1];
    const int c0 = sblk * seg;
    if (c0 >= nd) return;
    const int c1 = min(c0 + seg, nd);
    const int ntx = (m.nx + W::TX - 1) / W::TX;
    const int x0 = (tile % ntx) * W::TX, o0 = (tile / ntx) * W::TY;
    const int l = threadIdx.x, tx = l & 31, ty = l >> 5;
    const int x = x0 + tx, o = o0 + ty;
    const bool active = x < m.nx && o < no;
    const long long n = m.n;
    const long long sd = DIR == 1 ? (long long)m.nx : (long long)m.nx * m.ny;
    const long long so = DIR == 1 ? (long long)m.nx * m.ny : (long long)m.nx;
    const float *__restrict__ U = m.U32;
    const float *__restrict__ Q = (const float *)m.Q;
    float *ringI = smem;
    float *ringV = ringI + W::I_FLOATS;
    float *slab = ringV + W::V_FLOATS;
    // 16-byte copies when every row of the tile is whole and 16-byte aligned
    const bool vec = (m.nx % 4 == 0) && (x0 + W::TX <= m.nx);
    auto pmod = [](int c, int d) { return ((c % d) + d) % d; };

    // Copy items of this thread, fixed for the tile (only the plane offset changes):
    // 16-byte chunks of row r = (l >> 3) & 3, columns 4 (l & 7) .. + 3, fields
    // f = ty + 4 i of ring I and ring V; slab elements e = l + 128 i.
    constexpr int CI = (W::NI * W::TY * 8 + NL - 1) / NL, CV = (W::NVV * W::TY * 8 + NL - 1) / NL;
    constexpr int CS = (3 * W::NSL + NL - 1) / NL;
    const int vr = (l >> 3) & 3, vk = l & 7;
    const bool vrow = o0 + vr < no;
    const long long rowoff = (long long)(x0 + 4 * vk) + (long long)(o0 + vr) * so;
    const float *gI[CI];
    const float *gV[CV];
    const float *gS[CS];
#pragma unroll
    for (int i2 = 0; i2 < CI; ++i2) {
        const int f = ty + 4 * i2;
        const float *base = f < NV ? U + (long long)f * n
                                   : Q + (long long)(f == NV ? Q_U + DIR : (f == NV + 1 ? Q_P : Q_C)) * n;
        gI[i2] = f < W::NI ? base + rowoff : nullptr;
    }
#pragma unroll
    for (int i2 = 0; i2 < CV; ++i2) {
        const int f = ty + 4 * i2;
        gV[i2] = f < W::NVV ? Q + (long long)(Q_T + f) * n + rowoff : nullptr;
    }
#pragma unroll
    for (int i2 = 0; i2 < CS; ++i2) {
        const int e = l + NL * i2;
        if (e < 3 * W::NSL) {
            const int f = e / W::NSL, p = e - f * W::NSL;
            const int sy = p / W::SX, sx = p - sy * W::SX;
            int X = x0 - 1 + sx, O = o0 - 1 + sy;
            if ((unsigned)X >= (unsigned)m.nx) X = map_idx(X, m.nx, m.bc[0]);
            if ((unsigned)O >= (unsigned)no) O = map_idx(O, no, bco);
            gS[i2] = Q + (long long)f * n + (long long)X + (long long)O * so;
        } else {
            gS[i2] = nullptr;
        }
    }
    const int dvec = vr * W::TX + 4 * vk;

    auto stage_I = [&](int c) {
        const int cm = map_idx(c, nd, m.bc[DIR]);
        const long long plane = (long long)cm * sd;
        float *dst = ringI + pmod(c, W::DI) * W::NI * NL;
        if (vec) {
            if (vrow) {
#pragma unroll
                for (int i2 = 0; i2 < CI; ++i2)
                    if (gI[i2]) cp_async16(dst + (ty + 4 * i2) * NL + dvec, gI[i2] + plane);
            }
        } else if (active) {
            const long long cell = (long long)x + (long long)o * so + plane;
#pragma unroll
            for (int f = 0; f < W::NI; ++f) {
                const float *base = f < NV ? U + (long long)f * n
                                           : Q + (long long)(f == NV ? Q_U + DIR : (f == NV + 1 ? Q_P : Q_C)) * n;
                cp_async4(dst + f * NL + l, base + cell);
            }
        }
    };
    auto stage_V = [&](int c) {
        const int cm = map_idx(c, nd, m.bc[DIR]);
        const long long plane = (long long)cm * sd;
        const int slot = pmod(c, W::DV);
        float *dst = ringV + slot * W::NVV * NL;
        if (vec) {
            if (vrow) {
#pragma unroll
                for (int i2 = 0; i2 < CV; ++i2)
                    if (gV[i2]) cp_async16(dst + (ty + 4 * i2) * NL + dvec, gV[i2] + plane);
            }
        } else if (active) {
            const long long cell = (long long)x + (long long)o * so + plane;
            const float *qv = Q + (long long)Q_T * n;
#pragma unroll
            for (int f = 0; f < W::NVV; ++f) cp_async4(dst + f * NL + l, qv + (long long)f * n + cell);
        }
        float *sdst = slab + slot * 3 * W::NSL;
#pragma unroll
        for (int i2 = 0; i2 < CS; ++i2)
            if (gS[i2]) cp_async4(sdst + l + NL * i2, gS[i2] + plane);
    };

    stage_I(c0 - 2);
    stage_I(c0 - 1);
    stage_I(c0);
    stage_I(c0 + 1);
    stage_V(c0 - 1);
    stage_V(c0);
    cp_async_commit();

    const float ih = (float)m.invh[DIR];
    const long long lbase = (long long)x + (long long)o * so;
    const bool euler = m.stage_a == 0.0 && m.stage_b == 1.0;     // first RK stage: U^n not needed
    StageK sk;
    if (MODE == MODE_STAGE) sk = stage_k(m, m.clock[1]);
    float Gp[NV];
    for (int f = c0; f <= c1; ++f) {
        // the update's inputs of cell f-1, loaded before the wait so their latency overlaps it
        const bool upd = active && f > c0;
        const long long cell = lbase + (long long)(f - 1) * sd;
        float racc[NV];
        double uk[MODE == MODE_STAGE ? NV : 1], un[MODE == MODE_STAGE ? NV : 1];
        if (upd) {
            const float *__restrict__ rhs = (const float *)m.rhs;
#pragma unroll
            for (int v = 0; v < NV; ++v) racc[v] = rhs[v * n + cell];
            if (MODE == MODE_STAGE) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    uk[v] = m.U[v * n + cell];
                    un[v] = euler ? 0.0 : m.Un[v * n + cell];
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (f + 2 <= c1 + 1) stage_I(f + 2);
        cp_async_commit();
        WalkStencil<NS, DIR> st;
#pragma unroll
        for (int q = 0; q < 4; ++q) st.I[q] = ringI + pmod(f - 2 + q, W::DI) * W::NI * NL;
        st.V[0] = ringV + pmod(f - 1, W::DV) * W::NVV * NL;
        st.V[1] = ringV + pmod(f, W::DV) * W::NVV * NL;
        st.S[0] = slab + pmod(f - 1, W::DV) * 3 * W::NSL;
        st.S[1] = slab + pmod(f, W::DV) * 3 * W::NSL;
        st.l = l;
        st.sl = (ty + 1) * W::SX + tx + 1;
        float D[NV];
        if (active) face_visc<float, NS, DIR, false>(m, st, D);
        __syncthreads();
        if (f + 1 <= c1) stage_V(f + 1);
        cp_async_commit();
        if (active) {
            float Gn[NV], rl, rr;
            face_invisc<float, NS, DIR>(m, st, Gn, rl, rr);
            face_join<float, NS>(m, D, Gn);
            if (upd) {
                // as cell_update, from the preloaded inputs
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float L = fma(Gn[v] - Gp[v], ih, racc[v]);
                    if (MODE == MODE_ACCUM) ((float *)m.rhs)[v * n + cell] = L;
                    else if (MODE == MODE_RHS) m.dUdt[v * n + cell] = wide(L);
                    else m.Uout[v * n + cell] = stage_value(sk, L, uk[v], un[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) Gp[v] = Gn[v];
        }
    }
    cp_async_wait_all();
    __syncthreads();            // the rings are free for the block's next tile
}

// ----------------------------------------------------------------------------- staged x sweep (FP32 bulk)

// Each warp of a 128-thread block takes one row (fixed y, z) and walks it in chunks
// of 32 faces, lane l computing face F = F0 + l.  A chunk's window of 40 cells,
// starting at the 4-aligned cell 32 k - 4, is copied by cp.async, in field-rows:
//   I   fields: the NS + 4 conserved variables (FP32 copy), u, p, c;
//   V   fields: T, mu, lambda, X_s, Dc_s, h_s;
//   vel rows:   v, w of the row and (u, v) of rows y -+ 1, (u, w) of rows z -+ 1.
// The I rows are double-buffered per warp; the V and vel rows, read only by the
// viscous part of the face (at cells f-1 and f), have one 36-cell window per warp
// (starting 4 cells later in periodic rows, whose faces are shifted by one),
// refilled for the next chunk between the viscous and the inviscid part
// (warp-level synchronisation only): 44.5 KB per block of 4 warps, five blocks per SM.
// Periodic rows compute faces 1 .. nx (face nx has the stencil of face 0) and
// update cell 0 last; other rows compute faces 0 .. nx.
// Dynamic shared memory of a staged x-sweep block for ns species (as XTile<ns>::SMEM).
__host__ __device__ constexpr size_t x_staged_smem(int ns) {
    return sizeof(float) * (size_t)4 *
           ((size_t)2 * (ns + 7) * 40 + (size_t)(3 * ns + 13) * 36 + 16 + 2 * ((4 * ns + 21) / 2 * 2));
}

template <int NS>
struct XTile {
    static constexpr int WARPS = 4, WIN = 40, WINV = 36;
    static constexpr int NV = NS + 4, NI = NV + 3, NVV = 3 + 3 * NS, NVEL = 10;
    static constexpr int NFR = NI + NVV + NVEL;                // field-rows of a window
    static constexpr int BUF_I = NI * WIN, BUF_V = (NFR - NI) * WINV;
    static constexpr int WBUF = 2 * BUF_I + BUF_V;             // floats of one warp's buffers
    static constexpr int AUX = 16 + 2 * ((NFR + 1) / 2 * 2);    // floats per warp: G(1) stash, then NFR pointers
    static constexpr size_t SMEM = sizeof(float) * ((size_t)WARPS * WBUF + (size_t)WARPS * AUX);
    static_assert(SMEM == x_staged_smem(NS), "x_staged_smem out of step with XTile");
};

template <int NS>
struct XStencil {
    using X = XTile<NS>;
    const float *bi, *bv;    // I window; V / vel window less the offset of its start from the I window's
    int po;                  // I window position of the face's cell f-2
    __device__ __forceinline__ float at(int fr, int o) const {
        return fr < X::NI ? bi[fr * X::WIN + po + o] : bv[(fr - X::NI) * X::WINV + po + o];
    }
    __device__ __forceinline__ float u(int v, int o) const { return at(v, o); }
    __device__ __forceinline__ float q(int f, int o) const {
        if (f == Q_U) return at(X::NV + 0, o);
        if (f == Q_P) return at(X::NV + 1, o);
        if (f == Q_C) return at(X::NV + 2, o);
        if (f == Q_V) return at(X::NI + X::NVV + 0, o);
        if (f == Q_W) return at(X::NI + X::NVV + 1, o);
        return at(X::NI + f - Q_T, o);
    }
    __device__ __forceinline__ float qt(int f, int o, int t, bool plus) const {
        // vel rows 2..9: (u, v) at y-1, y+1, then (u, w) at z-1, z+1
        const int r = 2 + (t == 1 ? 0 : 4) + (plus ? 2 : 0) + (f == Q_U ? 0 : 1);
        return at(X::NI + X::NVV + r, o);
    }
};

template <int NS, int MODE>
__device__ __forceinline__ void sweep_x_staged_block(const MechDev &M, const Member &m, int blk, float *smem) {
    using X = XTile<NS>;
    constexpr int NV = NS + 4, WIN = X::WIN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = m.nx;
    const int nrows = m.ny * m.nz;
    const int row = blk * X::WARPS + warp;
    if (row >= nrows) return;                              // whole warp: no block-wide barrier below
    const int j = row % m.ny, k = row / m.ny;
    const long long n = m.n;
    const float *__restrict__ U = m.U32;
    const float *__restrict__ Q = (const float *)m.Q;
    float *bufI = smem + (size_t)warp * X::WBUF;           // two I buffers, then the V buffer
    float *bufV = bufI + 2 * X::BUF_I;
    float *stash = smem + (size_t)X::WARPS * X::WBUF + warp * X::AUX;
    const bool periodic = m.bc[0] == 0;
    const int fs = periodic ? 1 : 0;                       // first face computed
    const int nf = periodic ? nx : nx + 1;                 // faces fs .. fs + nf - 1
    const int nchunks = (nf + 31) / 32;
    const long long rowc = ((long long)k * m.ny + j) * nx;
    const int jm = map_idx(j - 1, m.ny, m.bc[1]), jp = map_idx(j + 1, m.ny, m.bc[1]);
    const int km = map_idx(k - 1, m.nz, m.bc[2]), kp = map_idx(k + 1, m.nz, m.bc[2]);
    const long long rjm = ((long long)k * m.ny + jm) * nx, rjp = ((long long)k * m.ny + jp) * nx;
    const long long rkm = ((long long)km * m.ny + j) * nx, rkp = ((long long)kp * m.ny + j) * nx;
    const bool vec_ok = nx % 4 == 0;

    // source of field-row fr (pointer to the row's cell 0), tabulated once per row
    auto src_of = [&](int fr) -> const float * {
        if (fr < NV) return U + (long long)fr * n + rowc;
        if (fr == NV) return Q + (long long)Q_U * n + rowc;
        if (fr == NV + 1) return Q + (long long)Q_P * n + rowc;
        if (fr == NV + 2) return Q + (long long)Q_C * n + rowc;
        if (fr < X::NI + X::NVV) return Q + (long long)(Q_T + fr - X::NI) * n + rowc;
        const int r = fr - X::NI - X::NVV;
        switch (r) {
            case 0: return Q + (long long)Q_V * n + rowc;
            case 1: return Q + (long long)Q_W * n + rowc;
            case 2: return Q + (long long)Q_U * n + rjm;
            case 3: return Q + (long long)Q_V * n + rjm;
            case 4: return Q + (long long)Q_U * n + rjp;
            case 5: return Q + (long long)Q_V * n + rjp;
            case 6: return Q + (long long)Q_U * n + rkm;
            case 7: return Q + (long long)Q_W * n + rkm;
            case 8: return Q + (long long)Q_U * n + rkp;
            default: return Q + (long long)Q_W * n + rkp;
        }
    };
    const float **tab = (const float **)(stash + 16) ;
    for (int fr = lane; fr < X::NFR; fr += 32) tab[fr] = src_of(fr);
    __syncwarp();
    // lanes 0..29 copy the window's 4-cell column chunk lane % 10 of field-rows
    // lane / 10, + 3, + 6, ...: the range test and any wrap are per lane, not per item
    // Window of chunk c: I rows from cell 32 c - 4 (40 cells), V / vel rows from
    // 32 c - 4 + vsh (36 cells).  Lane q + nq r copies the 4-cell column chunk q of
    // field-rows r, r + 3, r + 6, ... (nq = 10 chunks for I, 9 for V).
    const int vsh = periodic ? 4 : 0;
    const int sqI = lane % (WIN / 4), srI = lane / (WIN / 4);
    const int sqV = lane % (X::WINV / 4), srV = lane / (X::WINV / 4);
    const int sfrv = X::NI + srV;                          // the lane's first V / vel row
    // field-rows fr0, fr0 + 3, .. < fr1 into dst (row fr at dst + (fr - base) win), cells x0 + 4 q ..
    auto stage = [&](int x0, int q, int win, float *dst, int fr0, int fr1, int base) {
        const int x4 = x0 + 4 * q;
        float *dp = dst + (fr0 - base) * win + 4 * q;
        if (vec_ok && x4 >= 0 && x4 + 3 < nx) {
            for (int fr = fr0; fr < fr1; fr += 3, dp += 3 * win) cp_async16(dp, tab[fr] + x4);
        } else {
            int xi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xi[i] = map_idx(x4 + i, nx, m.bc[0]);
            for (int fr = fr0; fr < fr1; fr += 3, dp += 3 * win) {
                const float *sp = tab[fr];
#pragma unroll
                for (int i = 0; i < 4; ++i) cp_async4(dp + i, sp + xi[i]);
            }
        }
    };
    auto stage_I = [&](int c) {
        if (lane < 3 * (WIN / 4)) stage(32 * c - 4, sqI, WIN, bufI + (c & 1) * X::BUF_I, srI, X::NI, 0);
    };
    auto stage_V = [&](int c) {
        if (lane < 3 * (X::WINV / 4)) stage(32 * c - 4 + vsh, sqV, X::WINV, bufV, sfrv, X::NFR, X::NI);
    };

    const float ih = (float)m.invh[0];
    const bool euler = m.stage_a == 0.0 && m.stage_b == 1.0;     // first RK stage: U^n not needed
    StageK sk;
    if (MODE == MODE_STAGE) sk = stage_k(m, m.clock[1]);
    float Gc[NV];                      // lane 31's flux of the previous chunk
    stage_I(0);
    stage_V(0);
    cp_async_commit();
    for (int c = 0; c < nchunks; ++c) {
        const int F = fs + 32 * c + lane;
        const bool has_face = F < fs + nf;
        // this lane updates cell F - 1 (cell 0 of a periodic row comes last)
        const bool upd = has_face && F >= 1 && !(periodic && F == 1);
        const long long cell = rowc + (F - 1);
        float racc[NV];
        double uk[MODE == MODE_STAGE ? NV : 1], un[MODE == MODE_STAGE ? NV : 1];
        if (upd) {
            const float *__restrict__ rhs = (const float *)m.rhs;
#pragma unroll
            for (int v = 0; v < NV; ++v) racc[v] = rhs[v * n + cell];
            if (MODE == MODE_STAGE) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    uk[v] = m.U[v * n + cell];
                    un[v] = euler ? 0.0 : m.Un[v * n + cell];
                }
            }
        }
        cp_async_wait_all();
        __syncwarp();
        // the I buffer of chunk c + 1 is the one chunk c - 1 read
        if (c + 1 < nchunks) stage_I(c + 1);
        cp_async_commit();
        XStencil<NS> st;
        st.bi = bufI + (c & 1) * X::BUF_I;
        st.bv = bufV - vsh;
        st.po = F - 2 - (32 * c - 4);
        float D[NV];
        if (has_face) face_visc<float, NS, 0, false>(m, st, D);
        __syncwarp();
        if (c + 1 < nchunks) stage_V(c + 1);
        cp_async_commit();
        float G[NV];
        if (has_face) {
            float rl, rr;
            face_invisc<float, NS, 0>(m, st, G, rl, rr);
            face_join<float, NS>(m, D, G);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) G[v] = 0.f;
        }
        float Gl[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float up = __shfl_up_sync(0xffffffffu, G[v], 1);
            Gl[v] = lane == 0 ? Gc[v] : up;
            Gc[v] = __shfl_sync(0xffffffffu, G[v], 31);
        }
        if (periodic && c == 0 && lane == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) stash[v] = G[v];           // face 1, for cell 0
        }
        if (upd) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float L = fma(G[v] - Gl[v], ih, racc[v]);
                if (MODE == MODE_ACCUM) ((float *)m.rhs)[v * n + cell] = L;
                else if (MODE == MODE_RHS) m.dUdt[v * n + cell] = wide(L);
                else m.Uout[v * n + cell] = stage_value(sk, L, uk[v], un[v]);
            }
        }
        __syncwarp();
        if (periodic && F == nx) {
            // face nx = face 0: cell 0 from G(1) - G(nx)
            float dG[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) dG[v] = stash[v] - G[v];
            cell_update<float, NS, MODE>(m, rowc, dG, ih);
        }
        __syncwarp();
    }
    cp_async_wait_all();
}

template <int NS, int MODE>
__global__ void __launch_bounds__(128, 5) sweep_x_staged_kernel(int mslot, const __grid_constant__ Member m) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep_x_staged_block<NS, MODE>(M, m, blockIdx.x, (float *)smem_raw);
}

// Work tiles of a y / z sweep (128-thread blocks) and their dynamic shared memory.
template <typename R, int NS>
__host__ __device__ inline long long walk_tiles(int nx, int no) {
    if (sizeof(R) == 4) return (long long)((nx + WalkTile<NS>::TX - 1) / WalkTile<NS>::TX) * ((no + WalkTile<NS>::TY - 1) / WalkTile<NS>::TY);
    return ((long long)nx * no + 127) / 128;
}
template <typename R, int NS>
__host__ __device__ constexpr size_t walk_smem() { return sizeof(R) == 4 ? WalkTile<NS>::SMEM : 0; }

template <int NS, int DIR, int MODE>
__global__ void __launch_bounds__(128, MODE == MODE_STAGE ? 2 : 3) sweep_walk_staged_kernel(int mslot, const __grid_constant__ Member m, int seg) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep_walk_staged_block<NS, DIR, MODE>(M, m, blockIdx.x, blockIdx.y, seg, (float *)smem_raw);
}

// The source term plus the accumulated fluxes in the RHS buffer applied as the
// stage's output (MODE_RHS / MODE_STAGE) with no flux of its own: grids with no axis
// longer than one cell, and the stage update after sweeps that all accumulate.
template <typename R, int NS, int MODE>
__global__ void pointwise_final_kernel(const __grid_constant__ Member m) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= m.n) return;
    R z[NS + 4];
#pragma unroll
    for (int v = 0; v < NS + 4; ++v) z[v] = 0;
    cell_update<R, NS, MODE>(m, cell, z, R(0));
}

// ----------------------------------------------------------------------------- time step

// Step prologue: clock[2] = CFL, clock[3] = fixed dt (<= 0: rule), rate maxima cleared.
__global__ void step_params_kernel(double *clock, double cfl, double dt_fixed, unsigned long long *rates) {
    clock[2] = cfl;
    clock[3] = dt_fixed;
    rates[0] = 0ull;
    rates[1] = 0ull;
    rates[2] = 0ull;
}

// dt = min(CFL / acoustic, 0.25 h^2 / diffusive, 0.2 / chemical, laser clamp),
// or clock[3] if it is positive.
__global__ void dt_kernel(double *clock, const unsigned long long *rates, double hmin, int viscous, int chem,
                          int laser, double t0, double sigma_t, double *dt_out) {
    double dt = clock[3];
    if (!(dt > 0.0)) {
        const double ac = __longlong_as_double((long long)rates[0]);
        const double df = __longlong_as_double((long long)rates[1]);
        const double ch = __longlong_as_double((long long)rates[2]);
        dt = ac > 0.0 ? clock[2] / ac : 1.0e300;
        if (viscous && df > 0.0) dt = fmin(dt, 0.25 * hmin * hmin / df);
        if (chem && ch > 0.0) dt = fmin(dt, 0.2 / ch);
        if (laser) {
            const double t = clock[0];
            const double lo = t0 - 6.0 * sigma_t, hi = t0 + 6.0 * sigma_t;
            if (t + dt > lo && t < hi) dt = fmin(dt, fmax(0.25 * sigma_t, lo - t));
        }
    }
    clock[1] = dt;
    if (dt_out) *dt_out = dt;
}

__global__ void step_end_kernel(double *clock, double *t_out) {
    clock[0] += clock[1];
    if (t_out) *t_out = clock[0];
}

// ----------------------------------------------------------------------------- init state

template <int NS>
__global__ void init_state_kernel(int mslot, const double *__restrict__ prim, double *__restrict__ U,
                                  double *__restrict__ Tout, long long n) {
    const MechDev &M = c_mech[mslot];
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n) return;
    const double p = prim[cell], T = prim[n + cell];
    const double u = prim[2 * n + cell], v = prim[3 * n + cell], w = prim[4 * n + cell];
    double Y[NS], Rm = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Y[s] = prim[(5 + s) * n + cell];
        Rm = fma(Y[s], M.RW[s], Rm);
    }
    const double rho = p / (Rm * T);
    const int rng = nasa_range(M, T);
    const double invT = 1.0 / T;
    double e = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        U[s * n + cell] = rho * Y[s];
        e = fma(Y[s] * M.RW[s] * T, h_RT(M, rng, s, T, invT) - 1.0, e);
    }
    U[(NS + 0) * n + cell] = rho * u;
    U[(NS + 1) * n + cell] = rho * v;
    U[(NS + 2) * n + cell] = rho * w;
    U[(NS + 3) * n + cell] = rho * (e + 0.5 * (u * u + v * v + w * w));
    Tout[cell] = T;
}

// ----------------------------------------------------------------------------- diagnostics

// Per-block partial sums of U_v dV, HRR dV and the block max of T; a second
// kernel folds the partials in block order (deterministic).
template <int NS>
__global__ void __launch_bounds__(64) diag_kernel(int mslot, const __grid_constant__ Member m,
                                                   double *partial, int newton_maxit) {
    const MechDev &M = c_mech[mslot];
    constexpr int NV = NS + 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, tid = threadIdx.x;
    double *sC = (double *)smem_raw;
    double *sP = sC + NS * B;
    double *sRr = sP + NS * B;
    double *sW = sRr + NS * B;
    double *sD = sW + NS * B;
    __shared__ double red[NV + 2][64];
    const long long n = m.n, cell = (long long)blockIdx.x * B + tid;
    const double dV0 = m.h[0] * m.h[1] * m.h[2];
    double vals[NV + 2];
#pragma unroll
    for (int v = 0; v < NV + 2; ++v) vals[v] = 0.0;
    if (cell < n) {
        double rs[NS], Y[NS], rho = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rs[s] = m.U[s * n + cell];
            rho += rs[s];
        }
        const double irho = 1.0 / rho;
        const double u = m.U[NS * n + cell] * irho, v = m.U[(NS + 1) * n + cell] * irho, w = m.U[(NS + 2) * n + cell] * irho;
#pragma unroll
        for (int s = 0; s < NS; ++s) Y[s] = rs[s] * irho;
        const double e = m.U[(NS + 3) * n + cell] * irho - 0.5 * (u * u + v * v + w * w);
        double T = m.T[cell];
        MixPoly P;
        if (!newton_T<NS, true>(M, Y, e, T, newton_maxit, P)) flag_error(m, ST_NEWTON, cell);
        m.T[cell] = T;
        const int rng = nasa_range(M, T);
        const double invT = 1.0 / T, lnT = log(T);
        double hs[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) hs[s] = h_RT(M, rng, s, T, invT) * M.RW[s] * T;
        double hrr = 0.0;
        if (M.nr > 0) {
            chemistry_inputs<double, NS>(M, rng, rs, T, invT, lnT, sC + tid, sC + tid, sP + tid, sRr + tid, sW + tid,
                                         sD + tid, B, false);
            chemistry<double, NS>(M, T, lnT, invT, sC + tid, sC + tid, sP + tid, sRr + tid, sW + tid, sD + tid, B, false);
#pragma unroll
            for (int s = 0; s < NS; ++s) hrr -= hs[s] * sW[s * B + tid] * M.W[s];
        }
        const double dV = m.mapped ? m.gV[cell] : dV0;
#pragma unroll
        for (int v2 = 0; v2 < NV; ++v2) vals[v2] = m.U[v2 * n + cell] * dV;
        vals[NV] = hrr * dV;
        vals[NV + 1] = T;
    }
#pragma unroll
    for (int v = 0; v < NV + 2; ++v) red[v][tid] = vals[v];
    __syncthreads();
    if (tid < NV + 2) {
        double acc = 0.0;
        if (tid == NV + 1) {
            for (int q = 0; q < B; ++q) acc = fmax(acc, red[tid][q]);
        } else {
            for (int q = 0; q < B; ++q) acc += red[tid][q];
        }
        partial[(size_t)blockIdx.x * (NV + 2) + tid] = acc;
    }
}

// One warp per value: lane l folds partials l, l + 32, ... in order, then a fixed
// shuffle tree combines the lanes (the last value is a maximum).  Deterministic.
__global__ void diag_fold_kernel(const double *partial, int nblocks, int nvals, double *out) {
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (v >= nvals) return;
    const bool is_max = v == nvals - 1;
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double x = partial[(size_t)b * nvals + v];
        acc = is_max ? fmax(acc, x) : acc + x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, y) : acc + y;
    }
    if (lane == 0) out[v] = acc;
}

// ----------------------------------------------------------------------------- characteristic boundaries

// Navier-Stokes characteristic boundary conditions (NSCBC) for the reacting
// equations (Application examples: the diffusion flame's and the combustor's inflow
// and outflow boundaries, after Poinsot & Lele 1992 and Okong'o & Bellan 2002).
// Along an NSCBC axis the sweeps run with zero-gradient ghost cells; in the first and
// the last cell layer the scheme's inviscid normal term is then replaced by the
// characteristic form -P(V) d of the local one-dimensional inviscid relations:
//   wave amplitudes from one-sided second-order normal derivatives of
//   V = (rho, u_n, u_t1, u_t2, p, Y_s), c the frozen sound speed,
//     L1 = (u_n - c)(p' - rho c u_n'), L5 = (u_n + c)(p' + rho c u_n'),
//     L2 = u_n (c^2 rho' - p'), L3 = u_n u_t1', L4 = u_n u_t2', LY_s = u_n Y_s';
//   incoming amplitudes (speed pointing into the domain) replaced: at an outflow
//   side the acoustic one by K (p - p_inf), K = sigma c max(1 - M^2, 0) / ell, the
//   others by 0; at an inflow side by relaxations towards the target plane
//   (s eta_u rho c^2 max(1 - M^2, 0)(u_n - u_n,t) / ell, s = +1 low / -1 high;
//   -eta_T rho c Rbar (T - T_t) / ell; eta_t c (u_t - u_t,t) / ell;
//   eta_Y c (Y_s - Y_s,t) / ell);
//   d1 = (L2 + (L5 + L1) / 2) / c^2, d2 = (L5 + L1) / 2, d_n = (L5 - L1) / (2 rho c),
//   d_t1 = L3, d_t2 = L4, dY_s = LY_s (the rates -drho/dt, -dp/dt, -du/dt, -dY/dt);
//   conserved form with the multicomponent energy closure (e_s = h_s - R T / W_s,
//   gamma = rho c^2 / p):  [rho Y_s] -(Y_s d1 + rho dY_s);  [rho u_k] -(u_k d1 + rho d_k);
//   [E] -(|u|^2 d1 / 2 + rho u . d) + sum_s e_s [rho Y_s] + p / (gamma - 1)
//   (d1 / rho - d2 / p + Wbar sum_s dY_s / W_s).
// On a mapped grid the normal n is the boundary cell's mean area vector of the axis,
// S = (S_low + S_high) / 2, normalised, d/dn = (|S| / V) d/d(index), the shear amplitude
// is the vector u_n d(u - u_n n)/dn, and the metric part of the normal term,
// -(S_high - S_low) . F(U_b) / V, stays (a uniform flow stays at rest).
// One thread per boundary cell (both ends of the axis); it recomputes the cell's two
// inviscid face fluxes with the sweep's own face code and adds
// (characteristic term - scheme term) to the RHS accumulator, before the sweeps add
// the scheme term.  The characteristic term is formed in FP64 in both precisions
// (a few planes of cells).
struct NscbcSide {
    double p_inf, sigma, eta_u, eta_T, eta_t, eta_Y, ell;   // ell <= 0: the domain length
    const double *target;        // [4 + NS][plane] (u, v, w, T, Y_s) or nullptr (outflow)
};
struct NscbcAxis {
    NscbcSide s[2];              // low end, high end
};

template <typename R, typename UT, int NS, int DIR, int SCHEME, int GEOM>
__global__ void __launch_bounds__(128) nscbc_kernel(int mslot, const __grid_constant__ Member m,
                                                    const __grid_constant__ NscbcAxis bx) {
    constexpr int NV = NS + 4;
    constexpr int T1 = DIR == 0 ? 1 : 0, T2 = DIR == 2 ? 1 : 2;   // tangential axes, increasing
    const MechDev &M = c_mech[mslot];
    const int nn[3] = {m.nx, m.ny, m.nz};
    const int nd = nn[DIR], n1 = nn[T1];
    const long long plane = (long long)n1 * nn[T2];
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 2 * plane) return;
    const int side = id >= plane ? 1 : 0;
    const long long pc = id - side * plane;       // index on the boundary plane, t1 fastest
    int cc[3];
    cc[T1] = (int)(pc % n1);
    cc[T2] = (int)(pc / n1);
    cc[DIR] = side ? nd - 1 : 0;
    const long long st[3] = {1, m.nx, (long long)m.nx * m.ny};
    const long long n = m.n;
    const long long cell = (long long)cc[0] + (long long)cc[1] * st[1] + (long long)cc[2] * st[2];
    const long long inw = side ? -st[DIR] : st[DIR];
    const UT *U = (sizeof(UT) == 4) ? (const UT *)m.U32 : (const UT *)m.U;
    const R *Q = (const R *)m.Q;

    // boundary normal n and d/dn = kappa d/d(index): the axis and 1/h on a Cartesian
    // grid; on a mapped grid the cell's mean area vector of the axis, normalised, and
    // |S| / V, with dS = S_high - S_low for the metric part of the normal term
    double nv[3] = {0.0, 0.0, 0.0}, dS[3] = {0.0, 0.0, 0.0}, kappa;
    R Slo[3], Shi[3];
    if (GEOM) {
        int cf[3] = {cc[0], cc[1], cc[2]};
        const R *__restrict__ gS = (const R *)m.gS[DIR];
        const long long nf = face_count<DIR>(m);
        const long long f0 = face_index<DIR>(m, cf);
        cf[DIR] += 1;
        const long long f1 = face_index<DIR>(m, cf);
        double Sm2 = 0.0, Sb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Slo[k] = gS[k * nf + f0];
            Shi[k] = gS[k * nf + f1];
            Sb[k] = 0.5 * (wide(Slo[k]) + wide(Shi[k]));
            dS[k] = wide(Shi[k]) - wide(Slo[k]);
            Sm2 = fma(Sb[k], Sb[k], Sm2);
        }
        const double Sm = sqrt(Sm2);
#pragma unroll
        for (int k = 0; k < 3; ++k) nv[k] = Sb[k] / Sm;
        kappa = Sm / m.gV[cell];
    } else {
        nv[DIR] = 1.0;
        kappa = m.invh[DIR];
    }

    // the scheme's inviscid normal term, G at the cell's low face and high face
    R G0[NV], G1[NV];
    {
        R rl, rr;
        int cf[3] = {cc[0], cc[1], cc[2]};
        if (GEOM) {
            const double *__restrict__ gV = m.gV;
            if (SCHEME == 1) {
                const GlobalStencil6<R, UT, DIR> s0(m, U, Q, cf);
                face_invisc_teno_mapped<R, NS, DIR>(m, s0, Slo, G0, rl, rr);
                cf[DIR] += 1;
                const GlobalStencil6<R, UT, DIR> s1(m, U, Q, cf);
                face_invisc_teno_mapped<R, NS, DIR>(m, s1, Shi, G1, rl, rr);
            } else {
                const GlobalStencil<R, UT, DIR> s0(m, U, Q, cf);
                const R S0 = sqrt(Slo[0] * Slo[0] + Slo[1] * Slo[1] + Slo[2] * Slo[2]);
                const R h0 = narrow<R>(0.5 * (gV[s0.id[1]] + gV[s0.id[2]])) / S0;
                face_invisc_mapped<R, NS, DIR>(m, s0, Slo, h0 * h0 * R(1.0 / 3.0), G0, rl, rr);
                cf[DIR] += 1;
                const GlobalStencil<R, UT, DIR> s1(m, U, Q, cf);
                const R S1 = sqrt(Shi[0] * Shi[0] + Shi[1] * Shi[1] + Shi[2] * Shi[2]);
                const R h1 = narrow<R>(0.5 * (gV[s1.id[1]] + gV[s1.id[2]])) / S1;
                face_invisc_mapped<R, NS, DIR>(m, s1, Shi, h1 * h1 * R(1.0 / 3.0), G1, rl, rr);
            }
        } else if (SCHEME == 1) {
            const GlobalStencil6<R, UT, DIR> s0(m, U, Q, cf);
            face_invisc_teno<R, NS, DIR>(m, s0, G0, rl, rr);
            cf[DIR] += 1;
            const GlobalStencil6<R, UT, DIR> s1(m, U, Q, cf);
            face_invisc_teno<R, NS, DIR>(m, s1, G1, rl, rr);
        } else {
            const GlobalStencil<R, UT, DIR> s0(m, U, Q, cf);
            face_invisc<R, NS, DIR>(m, s0, G0, rl, rr);
            cf[DIR] += 1;
            const GlobalStencil<R, UT, DIR> s1(m, U, Q, cf);
            face_invisc<R, NS, DIR>(m, s1, G1, rl, rr);
        }
    }

    // primitives of the boundary cell and its two inward neighbours
    const double *__restrict__ Ud = m.U;
    double rho[3], u[3][3], p[3];                 // u[k][j]: component k, j cells inward
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long cj = cell + j * inw;
        double r = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) r += Ud[s * n + cj];
        rho[j] = r;
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k][j] = wide(Q[(Q_U + k) * n + cj]);
        p[j] = wide(Q[Q_P * n + cj]);
    }
    // d/dn = h2 (-3 f_0 + 4 f_1 - f_2), f_j j cells inward (h2 = -+kappa / 2 high / low)
    const double h2 = (side ? -0.5 : 0.5) * kappa;
    auto ddn = [&](const double (&f)[3]) { return h2 * (fma(-3.0, f[0], 4.0 * f[1]) - f[2]); };
    const double r0 = rho[0], p0 = p[0];
    const double ub[3] = {u[0][0], u[1][0], u[2][0]};
    const double u_n = nv[0] * ub[0] + nv[1] * ub[1] + nv[2] * ub[2];
    const double c = wide(Q[Q_C * n + cell]), T = wide(Q[Q_T * n + cell]);
    const double ir[3] = {1.0 / rho[0], 1.0 / rho[1], 1.0 / rho[2]};
    double Yb[NS], LY[NS];
    double iWbar = 0.0;                           // sum_s Y_s / W_s
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const double y[3] = {Ud[s * n + cell] * ir[0], Ud[s * n + cell + inw] * ir[1], Ud[s * n + cell + 2 * inw] * ir[2]};
        Yb[s] = y[0];
        LY[s] = u_n * ddn(y);
        iWbar = fma(y[0], M.invW[s], iWbar);
    }
    const double drho = ddn(rho), dp = ddn(p);
    double du[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) du[k] = ddn(u[k]);
    const double dun = nv[0] * du[0] + nv[1] * du[1] + nv[2] * du[2];
    double L1 = (u_n - c) * (dp - r0 * c * dun);
    double L5 = (u_n + c) * (dp + r0 * c * dun);
    double L2 = u_n * (c * c * drho - dp);
    double Lt[3];                                 // shear amplitude vector u_n d(u - u_n n)/dn
#pragma unroll
    for (int k = 0; k < 3; ++k) Lt[k] = u_n * fma(-dun, nv[k], du[k]);

    // incoming amplitudes
    const NscbcSide &sd = bx.s[side];
    const double ell = sd.ell > 0.0 ? sd.ell : (GEOM ? nd / kappa : nd * m.h[DIR]);
    const double F = fmax(1.0 - (u_n / c) * (u_n / c), 0.0);
    const double cl = c / ell;
    const bool tgt = sd.target != nullptr;
    double ac, ent = 0.0, sh[3] = {0.0, 0.0, 0.0};
    if (!tgt) {
        ac = sd.sigma * cl * F * (p0 - sd.p_inf);
    } else {
        const double *__restrict__ tg = sd.target;
        double tv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) tv[k] = tg[k * plane + pc];
        const double utn = nv[0] * tv[0] + nv[1] * tv[1] + nv[2] * tv[2];
        ac = (side ? -1.0 : 1.0) * sd.eta_u * r0 * c * cl * F * (u_n - utn);
        double Rbar = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) Rbar = fma(Yb[s], M.RW[s], Rbar);
        ent = -sd.eta_T * r0 * Rbar * cl * (T - tg[3 * plane + pc]);
#pragma unroll
        for (int k = 0; k < 3; ++k) sh[k] = sd.eta_t * cl * (fma(-u_n, nv[k], ub[k]) - fma(-utn, nv[k], tv[k]));
    }
    const bool in_m = side ? (u_n - c < 0.0) : (u_n - c > 0.0);
    const bool in_p = side ? (u_n + c < 0.0) : (u_n + c > 0.0);
    const bool in_0 = side ? (u_n < 0.0) : (u_n > 0.0);
    if (in_m) L1 = ac;
    if (in_p) L5 = ac;
    if (in_0) {
        L2 = ent;
#pragma unroll
        for (int k = 0; k < 3; ++k) Lt[k] = sh[k];
#pragma unroll
        for (int s = 0; s < NS; ++s) LY[s] = tgt ? sd.eta_Y * cl * (Yb[s] - sd.target[(4 + s) * plane + pc]) : 0.0;
    }

    // -P(V) d (velocity rate d_n n + Lt)
    const double d1 = (L2 + 0.5 * (L5 + L1)) / (c * c);
    const double d2 = 0.5 * (L5 + L1);
    const double dn = (L5 - L1) / (2.0 * r0 * c);
    double dv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dv[k] = fma(dn, nv[k], Lt[k]);
    double out[NV];
    double eW = 0.0, sdY = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        out[s] = -fma(Yb[s], d1, r0 * LY[s]);
        const double e_s = fma(-M.RW[s], T, wide(Q[(QL<NS>::H + s) * n + cell]));
        eW = fma(e_s, out[s], eW);
        sdY = fma(LY[s], M.invW[s], sdY);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) out[NS + k] = -fma(ub[k], d1, r0 * dv[k]);
    const double ke = 0.5 * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    const double gm1 = r0 * c * c / p0 - 1.0;
    const double dT = p0 / gm1 * (d1 / r0 - d2 / p0 + sdY / iWbar);
    out[NS + 3] = -(ke * d1 + r0 * (ub[0] * dv[0] + ub[1] * dv[1] + ub[2] * dv[2])) + eW + dT;
    if (GEOM) {
        // metric part of the normal term: -dS . F(U_b) / V
        const double iV = 1.0 / m.gV[cell];
        const double th = dS[0] * ub[0] + dS[1] * ub[1] + dS[2] * ub[2];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double f = th * Ud[v * n + cell];
            if (v >= NS && v < NS + 3) f = fma(p0, dS[v - NS], f);
            if (v == NS + 3) f = fma(p0, th, f);
            out[v] = fma(-f, iV, out[v]);
        }
    }

    R *__restrict__ rhs = (R *)m.rhs;
    const R ih = GEOM ? ((const R *)m.giV)[cell] : (R)m.invh[DIR];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double scheme = wide((G1[v] - G0[v]) * ih);
        rhs[v * n + cell] = narrow<R>(wide(rhs[v * n + cell]) + (out[v] - scheme));
    }
}

// ----------------------------------------------------------------------------- mapped-grid geometry

// Node (cell corner) coordinates X[3][nz+1][ny+1][nx+1] (FP64) -> the metric terms the
// mapped sweeps and cell state read.  Face area vector: half the cross product of the
// face's diagonals, oriented towards increasing index; cell volume: one third of the
// sum over its faces of the outward area vector dotted with the face centre; cell
// metric: the inverse of the matrix of dx/dxi_e, each column the mean of the cell's
// four edges along e; cell centre: the mean of its corners.  Computed in FP64.
struct Nodes {
    const double *X;
    int nx, ny, nz;
    long long nn;                 // (nx+1)(ny+1)(nz+1)
    __device__ __forceinline__ void at(int i, int j, int k, double (&p)[3]) const {
        const long long o = ((long long)k * (ny + 1) + j) * (nx + 1) + i;
        p[0] = X[o];
        p[1] = X[nn + o];
        p[2] = X[2 * nn + o];
    }
};

__device__ __forceinline__ void cross3(const double (&a)[3], const double (&b)[3], double (&c)[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// area vector and centre of face f of axis DIR at the other two indices (i, j, k with
// the DIR entry = f)
template <int DIR>
__device__ __forceinline__ void face_geom(const Nodes &N, int i, int j, int k, double (&S)[3], double (&c)[3]) {
    double p00[3], p11[3], pa[3], pb[3];
    if (DIR == 0) {
        N.at(i, j, k, p00); N.at(i, j + 1, k + 1, p11); N.at(i, j, k + 1, pa); N.at(i, j + 1, k, pb);
    } else if (DIR == 1) {
        N.at(i, j, k, p00); N.at(i + 1, j, k + 1, p11); N.at(i + 1, j, k, pa); N.at(i, j, k + 1, pb);
    } else {
        N.at(i, j, k, p00); N.at(i + 1, j + 1, k, p11); N.at(i, j + 1, k, pa); N.at(i + 1, j, k, pb);
    }
    double d1[3], d2[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        d1[q] = p11[q] - p00[q];
        d2[q] = pa[q] - pb[q];
        c[q] = 0.25 * (p00[q] + p11[q] + pa[q] + pb[q]);
    }
    cross3(d1, d2, S);
#pragma unroll
    for (int q = 0; q < 3; ++q) S[q] *= 0.5;
}

template <typename R, int DIR>
__global__ void geometry_face_kernel(const Nodes N, R *__restrict__ S) {
    const long long nf = DIR == 0 ? (long long)(N.nx + 1) * N.ny * N.nz
                                  : (DIR == 1 ? (long long)N.nx * (N.ny + 1) * N.nz : (long long)N.nx * N.ny * (N.nz + 1));
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nf) return;
    const int ax = DIR == 0 ? N.nx + 1 : N.nx, ay = DIR == 1 ? N.ny + 1 : N.ny;
    const int i = (int)(id % ax);
    const long long r = id / ax;
    const int j = (int)(r % ay), k = (int)(r / ay);
    double Sv[3], c[3];
    face_geom<DIR>(N, i, j, k, Sv, c);
#pragma unroll
    for (int q = 0; q < 3; ++q) S[q * nf + id] = narrow<R>(Sv[q]);
}

// cell volume, metric and centre; bad (if given) counts cells whose volume or metric
// determinant is not positive
template <typename R>
__global__ void geometry_cell_kernel(const Nodes N, R *__restrict__ Mo, double *__restrict__ Vo, R *__restrict__ iVo,
                                     double *__restrict__ C, unsigned long long *bad) {
    const long long n = (long long)N.nx * N.ny * N.nz;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int i = (int)(id % N.nx);
    const long long r = id / N.nx;
    const int j = (int)(r % N.ny), k = (int)(r / N.ny);
    double vol = 0.0, S[3], c[3];
    face_geom<0>(N, i + 1, j, k, S, c);
    vol += S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    face_geom<0>(N, i, j, k, S, c);
    vol -= S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    face_geom<1>(N, i, j + 1, k, S, c);
    vol += S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    face_geom<1>(N, i, j, k, S, c);
    vol -= S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    face_geom<2>(N, i, j, k + 1, S, c);
    vol += S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    face_geom<2>(N, i, j, k, S, c);
    vol -= S[0] * c[0] + S[1] * c[1] + S[2] * c[2];
    vol *= (1.0 / 3.0);
    double P[8][3];
#pragma unroll
    for (int q = 0; q < 8; ++q) N.at(i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2), P[q]);
    double A[3][3];                               // A[k][e] = d x_k / d xi_e
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        A[kk][0] = 0.25 * ((P[1][kk] - P[0][kk]) + (P[3][kk] - P[2][kk]) + (P[5][kk] - P[4][kk]) + (P[7][kk] - P[6][kk]));
        A[kk][1] = 0.25 * ((P[2][kk] - P[0][kk]) + (P[3][kk] - P[1][kk]) + (P[6][kk] - P[4][kk]) + (P[7][kk] - P[5][kk]));
        A[kk][2] = 0.25 * ((P[4][kk] - P[0][kk]) + (P[5][kk] - P[1][kk]) + (P[6][kk] - P[2][kk]) + (P[7][kk] - P[3][kk]));
    }
    // inverse by cofactors: Minv[e][k] = cof(A)[k][e] / det
    const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    const double id_ = 1.0 / det;
    double Mi[3][3];
    Mi[0][0] = c00 * id_;
    Mi[1][0] = c01 * id_;
    Mi[2][0] = c02 * id_;
    Mi[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id_;
    Mi[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id_;
    Mi[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id_;
    Mi[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id_;
    Mi[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id_;
    Mi[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id_;
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) Mo[(3 * e + kk) * n + id] = narrow<R>(Mi[e][kk]);
    Vo[id] = vol;
    iVo[id] = narrow<R>(1.0 / vol);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += P[q][kk];
        C[kk * n + id] = 0.125 * sum;
    }
    if (bad && !(vol > 0.0 && det > 0.0)) atomicAdd(bad, 1ull);
}

}  // namespace rf
