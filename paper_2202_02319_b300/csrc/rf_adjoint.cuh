// Discrete adjoint of the FP64 right-hand side (vector-Jacobian products).
//
// dU/dt = S(cell) + sum_d (G_d(f+1) - G_d(f)) / h_d, G = face flux of the cell
// fields Q (primitives, transport, enthalpies) and U.  Given lambda = dJ/d(dU/dt):
//   1. face adjoint: G_bar(f) = (lambda(f-1) - lambda(f)) / h_d; the hand-written
//      reverse of the face flux scatters into U_bar and Q_bar of the stencil cells
//      (FP64 atomics);
//   2. cell adjoint: U_bar(cell) += (dQ/dU)^T Q_bar + (dS/dU)^T lambda by a
//      hand-written reverse pass of the cell-state map (the temperature's adjoint
//      through one Newton step at the converged T: the implicit-function derivative).
// Parameter gradients (laser E, x0, y0, z0, sigma_r; ln A_j) are analytic.
// Non-smooth points take the subgradient of the forward branch: the LLF maximum
// goes to the stencil cell that attains it, |beta1 - beta0| has slope 0 at equality.
#pragma once

#include "rf_kernels.cuh"

namespace rf {

// 1/x in FP64: the Newton-Raphson rcp64 where x lies in the FP32 normal range (its
// seed's domain), a division elsewhere.
__device__ __forceinline__ double rcp_any(double x) {
    const double ax = fabs(x);
    return (ax > 1.0e-37 && ax < 1.0e37) ? rcp64(x) : 1.0 / x;
}


// ----------------------------------------------------------------------------- per-cell map

// Reverse (vector-Jacobian product) of the FP64 cell-state map U -> (Q, omega,
// HRR) in one pass: the forward values are recomputed, then
//   Ub += (dQ/dU)^T Qb + (d omega/dU)^T lamS + hb (dHRR/dU),
// where Qb(q) = Qbar[q * n + cell].  The temperature is one Newton
// step T = Tc - (e(Tc; Y) - e) / cv(Tc; Y) from the converged Tc, so its adjoint is
// the implicit-function derivative.  Species arrays indexed by the compact
// stoichiometry at run time (C, C G, 1/G and their adjoints) live in per-thread
// local memory.
template <int NS>
__device__ void cell_map_reverse(const MechDev &M, const double (&U)[NS + 4], double Tc, bool chem,
                                 const double *__restrict__ Qbar, long long n, long long cell,
                                 const double *__restrict__ lam, double hb, double (&Ub)[NS + 4]) {
    constexpr int NV = NS + 4;
    auto QB = [&](int q) { return Qbar[(size_t)q * n + cell]; };
    // ---------------------------------------------------------------- forward values
    double rho = U[0];
#pragma unroll
    for (int s = 1; s < NS; ++s) rho += U[s];
    const double irho = 1.0 / rho;
    const double u = U[NS] * irho, v = U[NS + 1] * irho, w = U[NS + 2] * irho;
    double Y[NS], Rm = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Y[s] = U[s] * irho;
        Rm += Y[s] * M.RW[s];
    }
    const double e = U[NS + 3] * irho - 0.5 * (u * u + v * v + w * w);
    const int rng = nasa_range(M, Tc);
    const double invTc = 1.0 / Tc;
    double es[NS], cvs[NS], em = 0.0, cvm = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        es[s] = (h_RT(M, rng, s, Tc, invTc) - 1.0) * M.RW[s] * Tc;
        cvs[s] = (cp_R<double>(M, rng, s, Tc) - 1.0) * M.RW[s];
        em += Y[s] * es[s];
        cvm += Y[s] * cvs[s];
    }
    const double icv = 1.0 / cvm, res = em - e;
    const double T = Tc - res * icv;
    const double invT = 1.0 / T;
    double cps[NS], cpm = 0.0, hs[NS], dhs[NS], dcps[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const double *a = M.cpc[rng][s];
        cps[s] = ((((T * a[4] + a[3]) * T + a[2]) * T + a[1]) * T + a[0]) * M.RW[s];
        dcps[s] = (((4.0 * a[4] * T + 3.0 * a[3]) * T + 2.0 * a[2]) * T + a[1]) * M.RW[s];
        cpm += Y[s] * cps[s];
        const double *c = M.ec[rng][s];
        const double Pe = (((T * c[4] + c[3]) * T + c[2]) * T + c[1]) * T + c[0];
        const double dPe = ((4.0 * c[4] * T + 3.0 * c[3]) * T + 2.0 * c[2]) * T + c[1];
        hs[s] = (Pe + invT * c[5]) * T * M.RW[s];            // = RW (T Pe(T) + c5)
        dhs[s] = (Pe + T * dPe) * M.RW[s];
    }
    const double cv = cpm - Rm;
    const double p = rho * Rm * T;
    const double r = cpm / cv;
    const double c = sqrt(r * Rm * T);
    const double irm = 1.0 / Rm;
    double X[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) X[s] = Y[s] * M.RW[s] * irm;
    const double lnTs = log(T * (1.0 / 300.0));
    double mus[NS], sq[NS], isq[NS], den[NS], xr[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        mus[s] = exp(lnTs * M.mu_exp[s]) * M.mu_ref[s];
        sq[s] = sqrt(mus[s]);
        isq[s] = rcp_any(sq[s]);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        double d = 0.0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const double a = sq[i] * isq[j] * M.wc[i][j] + 1.0;
            d += X[j] * (a * a) * M.wd[i][j];
        }
        den[i] = rcp_any(d);                    // 1 / sum_j X_j Phi_ij
        xr[i] = X[i] * den[i];
    }
    // ---------------------------------------------------------------- reverse
    double Yb[NS], Xb[NS], hsb[NS], cpsb[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Yb[s] = 0.0;
        Xb[s] = QB(QL<NS>::X + s);
        hsb[s] = QB(QL<NS>::H + s);
        cpsb[s] = 0.0;
    }
#pragma unroll
    for (int v2 = 0; v2 < NV; ++v2) Ub[v2] = 0.0;
    double Tb = QB(Q_T), pb = QB(Q_P), cb = QB(Q_C), ub = QB(Q_U), vb = QB(Q_V), wb = QB(Q_W);
    const double mub = QB(Q_MU), lamb = QB(Q_LAM);
    double rhob = 0.0, Rmb = 0.0, irhob = 0.0, lnTsb = 0.0, invTb = 0.0;
    // chemistry: omega_s = W_s sum_j nu_sj q_j, HRR = -sum_s h_s omega_s
    if (chem && M.nr > 0) {
        const double lnT = log(T);
        double G[NS], C[NS], sP[NS], sR[NS], sCb[NS], sPb[NS], sRb[NS], wd[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double *g = M.gc[rng][s];
            G[s] = exp((((T * g[4] + g[3]) * T + g[2]) * T + g[1]) * T + g[0] + invT * g[5] + lnT * g[6]);
            C[s] = U[s] * M.invW[s];
            sP[s] = C[s] * G[s];
            sR[s] = rcp_any(G[s]);
            sCb[s] = sPb[s] = sRb[s] = 0.0;
            wd[s] = 0.0;
        }
        // forward rates (omega needed for the HRR adjoint)
        for (int j = 0; j < M.nr; ++j) {
            const double kf = exp(lnT * M.b[j] - invT * M.Theta[j] + M.lnA[j]);
            double cf = kf;
            for (int k = 0; k < M.n_reac[j]; ++k) cf *= C[M.reac[j][k]];
            double q = cf;
            if (M.rev[j]) {
                double pr = kf;
                for (int k = 0; k < M.n_prod[j]; ++k) pr *= sP[M.prod[j][k]];
                for (int k = 0; k < M.n_reac[j]; ++k) pr *= sR[M.reac[j][k]];
                q -= pr;
            }
            for (int k = 0; k < M.n_net[j]; ++k) wd[M.net_sp[j][k]] += q * (double)M.net_nu[j][k];
        }
        double sWdb[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double Ws = wd[s] * M.W[s];
            hsb[s] -= hb * Ws;
            sWdb[s] = (lam[(size_t)s * n + cell] - hb * hs[s]) * M.W[s];
        }
        double lnTb = 0.0;
        for (int j = 0; j < M.nr; ++j) {
            double qb = 0.0;
            for (int k = 0; k < M.n_net[j]; ++k) qb += sWdb[M.net_sp[j][k]] * (double)M.net_nu[j][k];
            if (qb == 0.0) continue;
            const double kf = exp(lnT * M.b[j] - invT * M.Theta[j] + M.lnA[j]);
            const int nrc = M.n_reac[j], npd = M.n_prod[j];
            double prodC = 1.0;
            for (int k = 0; k < nrc; ++k) prodC *= C[M.reac[j][k]];
            double kfb = qb * prodC;
            for (int k = 0; k < nrc; ++k) {
                double part = qb * kf;
                for (int k2 = 0; k2 < nrc; ++k2)
                    if (k2 != k) part *= C[M.reac[j][k2]];
                sCb[M.reac[j][k]] += part;
            }
            if (M.rev[j]) {
                double prodR = 1.0;
                for (int k = 0; k < npd; ++k) prodR *= sP[M.prod[j][k]];
                for (int k = 0; k < nrc; ++k) prodR *= sR[M.reac[j][k]];
                kfb -= qb * prodR;
                for (int k = 0; k < npd; ++k) {
                    double part = -qb * kf;
                    for (int k2 = 0; k2 < npd; ++k2)
                        if (k2 != k) part *= sP[M.prod[j][k2]];
                    for (int k2 = 0; k2 < nrc; ++k2) part *= sR[M.reac[j][k2]];
                    sPb[M.prod[j][k]] += part;
                }
                for (int k = 0; k < nrc; ++k) {
                    double part = -qb * kf;
                    for (int k2 = 0; k2 < npd; ++k2) part *= sP[M.prod[j][k2]];
                    for (int k2 = 0; k2 < nrc; ++k2)
                        if (k2 != k) part *= sR[M.reac[j][k2]];
                    sRb[M.reac[j][k]] += part;
                }
            }
            const double zb = kfb * kf;
            lnTb += zb * M.b[j];
            invTb -= zb * M.Theta[j];
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double Gb = sPb[s] * C[s] - sRb[s] * sR[s] * sR[s];
            Ub[s] += (sCb[s] + sPb[s] * G[s]) * M.invW[s];
            const double lnGb = Gb * G[s];
            const double *g = M.gc[rng][s];
            Tb += lnGb * ((((4.0 * g[4] * T + 3.0 * g[3]) * T + 2.0 * g[2]) * T + g[1]));
            invTb += lnGb * g[5];
            lnTb += lnGb * g[6];
        }
        Tb += lnTb * invT;
    }
    // mixture-averaged diffusion: Dc_s = (rho / Wbar) D_s W_s
    if (NS > 1) {
        const double fT = exp(1.75 * lnTs) * PATM / p;
        double Xe[NS], Wbe = 0.0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            Xe[j] = X[j] + EPS_D;
            Wbe += Xe[j] * M.W[j];
        }
        const double rhoW = rho * Rm * (1.0 / RU);
        double rhoWb = 0.0, fTb = 0.0, Wbeb = 0.0, Xeb[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) Xeb[j] = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
            double num = 0.0, dd = 0.0;
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                if (j == s2) continue;
                num += Xe[j] * M.W[j];
                dd += Xe[j] * M.invDref[s2][j];
            }
            const double Dm = num * fT / (Wbe * dd);
            const double QDb = QB(QL<NS>::DC + s2);
            rhoWb += QDb * Dm * M.W[s2];
            const double t = QDb * rhoW * M.W[s2] * Dm;          // Dm_bar * Dm
            const double numb = t * rcp_any(num), ddb = -t * rcp_any(dd);
            fTb += t * rcp_any(fT);
            Wbeb -= t * rcp_any(Wbe);
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                if (j == s2) continue;
                Xeb[j] += numb * M.W[j] + ddb * M.invDref[s2][j];
            }
        }
#pragma unroll
        for (int j = 0; j < NS; ++j) Xb[j] += Xeb[j] + Wbeb * M.W[j];
        rhob += rhoWb * Rm * (1.0 / RU);
        Rmb += rhoWb * rho * (1.0 / RU);
        lnTsb += fTb * fT * 1.75;
        pb -= fTb * fT / p;
    }
    // Wilke viscosity and conductivity
    double sqb[NS], isqb[NS], musb[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) sqb[s] = isqb[s] = 0.0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const double fac = cps[i] + M.eucken[i];
        const double xrb = mub * mus[i] + lamb * mus[i] * fac;
        musb[i] = mub * xr[i] + lamb * xr[i] * fac;
        cpsb[i] += lamb * xr[i] * mus[i];
        Xb[i] += xrb * den[i];
        const double denb = -xrb * xr[i] * den[i];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const double a = sq[i] * isq[j] * M.wc[i][j] + 1.0;
            Xb[j] += denb * (a * a) * M.wd[i][j];
            const double ab = denb * X[j] * 2.0 * a * M.wd[i][j];
            sqb[i] += ab * isq[j] * M.wc[i][j];
            isqb[j] += ab * sq[i] * M.wc[i][j];
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        sqb[s] -= isqb[s] * isq[s] * isq[s];
        musb[s] += sqb[s] * 0.5 * isq[s];
        lnTsb += musb[s] * mus[s] * M.mu_exp[s];
    }
    Tb += lnTsb / T;
    // X_s = Y_s RW_s / Rm
    double irmb = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Yb[s] += Xb[s] * M.RW[s] * irm;
        irmb += Xb[s] * Y[s] * M.RW[s];
    }
    Rmb -= irmb * irm * irm;
    // c = sqrt(cpm / cv Rm T), p = rho Rm T, cv = cpm - Rm
    const double zb = cb * 0.5 / c;
    const double rb = zb * Rm * T;
    Rmb += zb * r * T;
    Tb += zb * r * Rm;
    double cpmb = rb / cv;
    const double cvb = -rb * r / cv;
    rhob += pb * Rm * T;
    Rmb += pb * rho * T;
    Tb += pb * rho * Rm;
    cpmb += cvb;
    Rmb -= cvb;
    // h_s(T), cp_s(T), cpm
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Tb += hsb[s] * dhs[s];
        Yb[s] += cpmb * cps[s];
        cpsb[s] += cpmb * Y[s];
        Tb += cpsb[s] * dcps[s];
    }
    Tb -= invTb * invT * invT;
    // T = Tc - (em - e) / cvm
    const double emb = -Tb * icv, eb = Tb * icv, cvmb = Tb * res * icv * icv;
#pragma unroll
    for (int s = 0; s < NS; ++s) Yb[s] += emb * es[s] + cvmb * cvs[s] + Rmb * M.RW[s];
    // e = E / rho - |u|^2 / 2
    Ub[NS + 3] += eb * irho;
    irhob += eb * U[NS + 3];
    ub -= eb * u;
    vb -= eb * v;
    wb -= eb * w;
    // Y, u, v, w, rho
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        Ub[s] += Yb[s] * irho;
        irhob += Yb[s] * U[s];
    }
    Ub[NS] += ub * irho;
    Ub[NS + 1] += vb * irho;
    Ub[NS + 2] += wb * irho;
    irhob += ub * U[NS] + vb * U[NS + 1] + wb * U[NS + 2];
    rhob -= irhob * irho * irho;
#pragma unroll
    for (int s = 0; s < NS; ++s) Ub[s] += rhob;
}

// Rate of progress q_j of every reaction at a cell (FP64 values), for the
// ln A_j gradients: d omega_s / d ln A_j = W_s nu_sj q_j.
template <int NS>
__device__ void rates_of_progress(const MechDev &M, const double (&rs)[NS], double T, double *qout, double *sG) {
    const int rng = nasa_range(M, T);
    const double invT = 1.0 / T, lnT = log(T);
    for (int s = 0; s < NS; ++s) sG[s] = exp(lnG(M, rng, s, T, invT, lnT));
    for (int j = 0; j < M.nr; ++j) {
        const double kf = exp(M.lnA[j] + M.b[j] * lnT - M.Theta[j] * invT);
        double cf = kf;
        for (int k = 0; k < M.n_reac[j]; ++k) cf *= rs[M.reac[j][k]] * M.invW[M.reac[j][k]];
        double q = cf;
        if (M.rev[j]) {
            double pr = kf;
            for (int k = 0; k < M.n_prod[j]; ++k) {
                const int s = M.prod[j][k];
                pr *= rs[s] * M.invW[s] * sG[s];
            }
            for (int k = 0; k < M.n_reac[j]; ++k) pr /= sG[M.reac[j][k]];
            q -= pr;
        }
        qout[j] = q;
    }
}

// ----------------------------------------------------------------------------- cell adjoint

// U_bar(cell) += (dQ/dU)^T Q_bar + (d omega/dU)^T lambda_species + wH (dHRR/dU) dV;
// grads[5 + j] += sum_s (lambda_s + wH dV (-h_s)) W_s nu_sj q_j (ln A_j);
// grads[0..4] += lambda_E dq_L/d(E, x0, y0, z0, sigma_r).
template <int NS>
__global__ void __launch_bounds__(64) adjoint_cell_kernel(int mslot, const __grid_constant__ Member m,
                                                          const double *__restrict__ Qbar, const double *__restrict__ lam,
                                                          double *__restrict__ Ubar, double *__restrict__ grads,
                                                          double wH) {
    const MechDev &M = c_mech[mslot];
    constexpr int NV = NS + 4;
    const long long n = m.n;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double red[5 + NRMAX][64];
    double gl[5 + NRMAX];
    for (int q = 0; q < 5 + NRMAX; ++q) gl[q] = 0.0;
    const bool chem = !(m.flags & F_NO_CHEM);
    const double dV = m.h[0] * m.h[1] * m.h[2];
    if (cell < n) {
        double Uv[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Uv[v] = m.U[v * n + cell];
        const double Tc = m.T[cell];
        double Ub[NV];
        cell_map_reverse<NS>(M, Uv, Tc, chem, Qbar, n, cell, lam, wH * dV, Ub);
#pragma unroll
        for (int v = 0; v < NV; ++v) Ubar[(size_t)v * n + cell] += Ub[v];
        // parameter gradients
        if (chem && M.nr > 0) {
            double rs[NS], qj[NRMAX], sG[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) rs[s] = Uv[s];
            rates_of_progress<NS>(M, rs, Tc, qj, sG);
            const int rng = nasa_range(M, Tc);
            double cw[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s)
                cw[s] = (lam[(size_t)s * n + cell] - wH * dV * h_RT(M, rng, s, Tc, 1.0 / Tc) * M.RW[s] * Tc) * M.W[s];
            for (int j = 0; j < M.nr; ++j) {
                double a = 0.0;
                for (int k = 0; k < M.n_net[j]; ++k) a += cw[M.net_sp[j][k]] * (double)M.net_nu[j][k];
                gl[5 + j] = a * qj[j];
            }
        }
        if (m.laser_on && !(m.flags & F_NO_LASER)) {
            const long long nxy = (long long)m.nx * m.ny;
            const int k = (int)(cell / nxy);
            const long long rem = cell - (long long)k * nxy;
            const int j = (int)(rem / m.nx), i = (int)(rem - (long long)j * m.nx);
            const double t = m.t_host;
            const double sr = m.las[4], st = m.las[6];
            const double dx = (i + 0.5) * m.h[0] - m.las[1], dy = (j + 0.5) * m.h[1] - m.las[2];
            double dz = 0.0, dims = 2.0;
            if (m.nz > 1) {
                dz = (k + 0.5) * m.h[2] - m.las[3];
                dims = 3.0;
            }
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double tt = (t - m.las[5]) / st;
            const double two_pi = 6.283185307179586;
            const double norm = m.nz == 1 ? m.las[0] / (two_pi * sqrt(two_pi) * sr * sr * st)
                                          : m.las[0] / (two_pi * two_pi * sr * sr * sr * st);
            const double qL = norm * exp(-0.5 * tt * tt) * exp(-0.5 * r2 / (sr * sr));
            const double lE = lam[(size_t)(NS + 3) * n + cell];
            gl[0] = lE * qL / m.las[0];
            gl[1] = lE * qL * dx / (sr * sr);
            gl[2] = lE * qL * dy / (sr * sr);
            gl[3] = m.nz > 1 ? lE * qL * dz / (sr * sr) : 0.0;
            gl[4] = lE * qL * (r2 / (sr * sr * sr) - dims / sr);
        }
    }
    // block reduction in fixed order, one atomic per block and parameter
    const int np = 5 + M.nr;
    for (int q = 0; q < np; ++q) red[q][threadIdx.x] = gl[q];
    __syncthreads();
    if (threadIdx.x < np) {
        double a = 0.0;
        for (int t = 0; t < blockDim.x; ++t) a += red[threadIdx.x][t];
        if (a != 0.0) atomicAdd(&grads[threadIdx.x], a);
    }
}

// ----------------------------------------------------------------------------- face adjoint

// Reverse of weno3z(a, b, c, e2): adds wbar * dW/d(a, b, c) into (ga, gb, gc), the
// grid-scaled eps = e2 (a^2 + b^2 + c^2) + EPS_WENO included.  Without the eps path
// the three derivatives sum to wbar (a common shift of a, b, c shifts W by as much);
// the eps path's share of that sum, epsb (a + b + c) with epsb = wbar dW/d eps 2 e2,
// is added to seps, so that callers can use the shift identity exactly.
__device__ __forceinline__ void weno3z_adj(double a, double b, double c, double e2, double wbar, double &ga, double &gb,
                                           double &gc, double &seps) {
    // w = q1 + omega0 (q0 - q1), q0 - q1 = (d0 - d1) / 2: every factor of the
    // reverse pass is a difference of f (no q - w of O(f) values that cancel)
    const double d0 = b - a, d1 = c - b;
    const double dq = 0.5 * (d0 - d1);
    const double b0 = d0 * d0, b1 = d1 * d1;
    const double tau = fabs(b1 - b0);
    const double eps = fma(e2, fma(a, a, fma(b, b, c * c)), EPS_WENO);
    const double e0 = b0 + eps, e1 = b1 + eps;
    // three reciprocals instead of ten divisions (FP64 divisions are long sequences on
    // the FP64 pipe, which bounds this kernel)
    const double ie0 = rcp_any(e0), ie1 = rcp_any(e1);
    const double te0 = tau * ie0, te1 = tau * ie1;
    const double al0 = (1.0 / 3.0) * (1.0 + te0), al1 = (2.0 / 3.0) * (1.0 + te1);
    const double S = al0 + al1, iS = rcp_any(S);
    const double om0 = al0 * iS, om1 = al1 * iS;
    const double dqb = wbar * om0, om0b = wbar * dq;
    const double al0b = om0b * om1 * iS, al1b = -om0b * om0 * iS;
    const double taub = al0b * (1.0 / 3.0) * ie0 + al1b * (2.0 / 3.0) * ie1;
    const double sg = b1 > b0 ? 1.0 : (b1 < b0 ? -1.0 : 0.0);
    const double e0b = -al0b * (1.0 / 3.0) * te0 * ie0, e1b = -al1b * (2.0 / 3.0) * te1 * ie1;
    const double b0b = e0b - sg * taub;
    const double b1b = e1b + sg * taub;
    const double epsb2 = 2.0 * e2 * (e0b + e1b);
    const double d0b = 0.5 * dqb + 2.0 * d0 * b0b;
    const double d1b = -0.5 * dqb + 2.0 * d1 * b1b;
    ga += -d0b + epsb2 * a;
    gb += 0.5 * wbar + d0b - d1b + epsb2 * b;
    gc += 0.5 * wbar + d1b + epsb2 * c;
    seps += epsb2 * ((a + b) + c);
}

// One face of axis DIR per thread: face f (left face of cell f) with
// G_bar = (lambda(L) - lambda(R)) / h, L = f - 1, R = f (a side outside the grid
// of a zero-gradient axis has no RHS and contributes nothing).
template <int NS, int DIR>
__global__ void __launch_bounds__(128) adjoint_face_kernel(const __grid_constant__ Member m, const double *__restrict__ lam,
                                                           double *__restrict__ Ubar, double *__restrict__ Qbar) {
    constexpr int NV = NS + 4;
    const long long n = m.n;
    const int nd = DIR == 0 ? m.nx : (DIR == 1 ? m.ny : m.nz);
    const bool periodic = m.bc[DIR] == 0;
    const int nf = periodic ? nd : nd + 1;
    const int n0 = DIR == 0 ? m.ny : m.nx;            // the two other axes
    const int n1 = DIR == 2 ? m.ny : m.nz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)nf * n0 * n1) return;
    const int f = (int)(gid % nf);
    const long long rest = gid / nf;
    const int a0 = (int)(rest % n0), a1 = (int)(rest / n0);
    int cc[3];
    cc[DIR] = f;
    if (DIR == 0) {
        cc[1] = a0;
        cc[2] = a1;
    } else if (DIR == 1) {
        cc[0] = a0;
        cc[2] = a1;
    } else {
        cc[0] = a0;
        cc[1] = a1;
    }
    const long long st[3] = {1, m.nx, (long long)m.nx * m.ny};
    const long long base = (long long)cc[0] * st[0] + (long long)cc[1] * st[1] + (long long)cc[2] * st[2] -
                           (long long)cc[DIR] * st[DIR];
    long long id[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) id[o] = base + (long long)map_idx(f + o - 2, nd, m.bc[DIR]) * st[DIR];
    const double ih = m.invh[DIR];
    const bool hasL = periodic || f >= 1, hasR = periodic || f < nd;
    const long long cL = id[1], cR = id[2];
    double Gb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double lL = hasL ? lam[(size_t)v * n + cL] : 0.0;
        const double lR = hasR ? lam[(size_t)v * n + cR] : 0.0;
        Gb[v] = (lL - lR) * ih;
    }
    const double *Q = (const double *)m.Q;
    const double *U = m.U;
    auto addQ = [&](int field, long long cell, double x) {
        if (x != 0.0) atomicAdd(&Qbar[(size_t)field * n + cell], x);
    };
    auto addU = [&](int var, long long cell, double x) {
        if (x != 0.0) atomicAdd(&Ubar[(size_t)var * n + cell], x);
    };
    double rhoL = 0.0, rhoR = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        rhoL += U[(size_t)s * n + cL];
        rhoR += U[(size_t)s * n + cR];
    }
    if (!(m.flags & F_NO_INVISCID)) {
        double un[4], pp[4], cs[4], unb[4] = {0, 0, 0, 0}, ppb[4] = {0, 0, 0, 0};
        double alpha = 0.0;
        int amax = 0;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            un[o] = Q[(size_t)(Q_U + DIR) * n + id[o]];
            pp[o] = Q[(size_t)Q_P * n + id[o]];
            cs[o] = Q[(size_t)Q_C * n + id[o]];
            const double l = fabs(un[o]) + cs[o];
            if (o == 0 || l > alpha) {
                alpha = l;
                amax = o;
            }
        }
        double alphab = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double Uv[4], fp[4], fm[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                Uv[o] = U[(size_t)v * n + id[o]];
                double F = un[o] * Uv[o];
                if (v == NS + DIR) F += pp[o];
                if (v == NS + 3) F += pp[o] * un[o];
                fp[o] = 0.5 * (F + alpha * Uv[o]);
                fm[o] = 0.5 * (F - alpha * Uv[o]);
            }
            double fpb[4] = {0, 0, 0, 0}, fmb[4] = {0, 0, 0, 0}, sp = 0.0, sm = 0.0;
            weno3z_adj(fp[0], fp[1], fp[2], m.weps[DIR], -Gb[v], fpb[0], fpb[1], fpb[2], sp);
            weno3z_adj(fm[3], fm[2], fm[1], m.weps[DIR], -Gb[v], fmb[3], fmb[2], fmb[1], sm);
            // d Fhat / d alpha = (Uhat+ - Uhat-) / 2 is a difference of two
            // reconstructions; apart from the eps path the partial derivatives of each
            // reconstruction sum to its weight, so a reference value U_L can be taken
            // out of the sum exactly, which keeps it free of cancellation between O(U)
            // terms; the eps paths' share (sp, sm) is added back with U_L.
            alphab += 0.5 * Uv[1] * (sp - sm);
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const double Fb = 0.5 * (fpb[o] + fmb[o]);
                double Ub = 0.5 * alpha * (fpb[o] - fmb[o]) + un[o] * Fb;
                alphab += 0.5 * (Uv[o] - Uv[1]) * (fpb[o] - fmb[o]);
                unb[o] += Uv[o] * Fb;
                if (v == NS + DIR) ppb[o] += Fb;
                if (v == NS + 3) {
                    ppb[o] += un[o] * Fb;
                    unb[o] += pp[o] * Fb;
                }
                addU(v, id[o], Ub);
            }
        }
        unb[amax] += alphab * (un[amax] > 0.0 ? 1.0 : (un[amax] < 0.0 ? -1.0 : 0.0));
        addQ(Q_C, id[amax], alphab);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            addQ(Q_U + DIR, id[o], unb[o]);
            addQ(Q_P, id[o], ppb[o]);
        }
    }
    if (!(m.flags & F_NO_VISCOUS)) {
        double velL[3], velR[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            velL[q] = Q[(size_t)(Q_U + q) * n + cL];
            velR[q] = Q[(size_t)(Q_U + q) * n + cR];
        }
        const double mu = 0.5 * (Q[(size_t)Q_MU * n + cL] + Q[(size_t)Q_MU * n + cR]);
        const double lamf = 0.5 * (Q[(size_t)Q_LAM * n + cL] + Q[(size_t)Q_LAM * n + cR]);
        double dn[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) dn[q] = (velR[q] - velL[q]) * ih;
        double dtd[3] = {0, 0, 0}, dtt[3] = {0, 0, 0};
        long long op[3] = {0, 0, 0}, om[3] = {0, 0, 0};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == DIR) continue;
            const int nt = t == 0 ? m.nx : (t == 1 ? m.ny : m.nz);
            op[t] = (long long)(map_idx(cc[t] + 1, nt, m.bc[t]) - cc[t]) * st[t];
            om[t] = (long long)(map_idx(cc[t] - 1, nt, m.bc[t]) - cc[t]) * st[t];
            const double q4 = 0.25 * m.invh[t];
            const double *vd = Q + (size_t)(Q_U + DIR) * n;
            const double *vt = Q + (size_t)(Q_U + t) * n;
            dtd[t] = ((vd[cL + op[t]] - vd[cL + om[t]]) + (vd[cR + op[t]] - vd[cR + om[t]])) * q4;
            dtt[t] = ((vt[cL + op[t]] - vt[cL + om[t]]) + (vt[cR + op[t]] - vt[cR + om[t]])) * q4;
        }
        double div = dn[DIR];
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t != DIR) div += dtt[t];
        double tau[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) tau[q] = q == DIR ? mu * (2.0 * dn[DIR]) - (2.0 / 3.0) * mu * div : mu * (dtd[q] + dn[q]);
        double dX[NS], Dcf[NS], Yf[NS], hf[NS], YL[NS], YR[NS];
        double corr = 0.0;
        const double irL = rcp_any(rhoL), irR = rcp_any(rhoR);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            dX[s] = (Q[(size_t)(QL<NS>::X + s) * n + cR] - Q[(size_t)(QL<NS>::X + s) * n + cL]) * ih;
            Dcf[s] = 0.5 * (Q[(size_t)(QL<NS>::DC + s) * n + cL] + Q[(size_t)(QL<NS>::DC + s) * n + cR]);
            YL[s] = U[(size_t)s * n + cL] * irL;
            YR[s] = U[(size_t)s * n + cR] * irR;
            Yf[s] = 0.5 * (YL[s] + YR[s]);
            hf[s] = 0.5 * (Q[(size_t)(QL<NS>::H + s) * n + cL] + Q[(size_t)(QL<NS>::H + s) * n + cR]);
            corr += Dcf[s] * dX[s];
        }
        double J[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) J[s] = -Dcf[s] * dX[s] + Yf[s] * corr;
        // reverse
        const double qbar = -Gb[NS + 3], workb = Gb[NS + 3];
        double taub[3], ufb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            taub[k] = Gb[NS + k] + workb * 0.5 * (velL[k] + velR[k]);
            ufb[k] = workb * tau[k];
        }
        double velLb[3], velRb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) velLb[k] = velRb[k] = 0.5 * ufb[k];
        const double TL = Q[(size_t)Q_T * n + cL], TR = Q[(size_t)Q_T * n + cR];
        const double lamb = -qbar * (TR - TL) * ih;
        addQ(Q_T, cR, -qbar * lamf * ih);
        addQ(Q_T, cL, qbar * lamf * ih);
        addQ(Q_LAM, cL, 0.5 * lamb);
        addQ(Q_LAM, cR, 0.5 * lamb);
        double Jb[NS], corrb = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            Jb[s] = -Gb[s] + qbar * hf[s];
            const double hfb = qbar * J[s];
            addQ(QL<NS>::H + s, cL, 0.5 * hfb);
            addQ(QL<NS>::H + s, cR, 0.5 * hfb);
            corrb += Jb[s] * Yf[s];
        }
        double YLb[NS], YRb[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double Dcfb = -Jb[s] * dX[s] + corrb * dX[s];
            const double dXb = -Jb[s] * Dcf[s] + corrb * Dcf[s];
            const double Yfb = Jb[s] * corr;
            addQ(QL<NS>::DC + s, cL, 0.5 * Dcfb);
            addQ(QL<NS>::DC + s, cR, 0.5 * Dcfb);
            addQ(QL<NS>::X + s, cR, dXb * ih);
            addQ(QL<NS>::X + s, cL, -dXb * ih);
            YLb[s] = YRb[s] = 0.5 * Yfb;
        }
        // Y_s = U_s / rho: dY_s/dU_k = (delta_sk - Y_s) / rho
        double sL = 0.0, sR = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            sL += YLb[s] * YL[s];
            sR += YRb[s] * YR[s];
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            addU(s, cL, (YLb[s] - sL) * irL);
            addU(s, cR, (YRb[s] - sR) * irR);
        }
        double mub = 0.0, dnb[3] = {0, 0, 0}, dtdb[3] = {0, 0, 0}, dttb[3] = {0, 0, 0}, divb = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (q == DIR) {
                mub += taub[q] * (2.0 * dn[DIR] - (2.0 / 3.0) * div);
                dnb[DIR] += taub[q] * 2.0 * mu;
                divb += -taub[q] * (2.0 / 3.0) * mu;
            } else {
                mub += taub[q] * (dtd[q] + dn[q]);
                dtdb[q] += taub[q] * mu;
                dnb[q] += taub[q] * mu;
            }
        }
        dnb[DIR] += divb;
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t != DIR) dttb[t] += divb;
        addQ(Q_MU, cL, 0.5 * mub);
        addQ(Q_MU, cR, 0.5 * mub);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            velRb[q] += dnb[q] * ih;
            velLb[q] -= dnb[q] * ih;
            addQ(Q_U + q, cL, velLb[q]);
            addQ(Q_U + q, cR, velRb[q]);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == DIR) continue;
            const double q4 = 0.25 * m.invh[t];
            const double gd = dtdb[t] * q4, gt = dttb[t] * q4;
            addQ(Q_U + DIR, cL + op[t], gd);
            addQ(Q_U + DIR, cL + om[t], -gd);
            addQ(Q_U + DIR, cR + op[t], gd);
            addQ(Q_U + DIR, cR + om[t], -gd);
            addQ(Q_U + t, cL + op[t], gt);
            addQ(Q_U + t, cL + om[t], -gt);
            addQ(Q_U + t, cR + op[t], gt);
            addQ(Q_U + t, cR + om[t], -gt);
        }
    }
}

// y = a x + b y over n values
__global__ void axpby_kernel(double *__restrict__ y, const double *__restrict__ x, double a, double b, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], b * y[i]);
}

}  // namespace rf
