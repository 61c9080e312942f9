// C ABI of the reacting-flow RHS library (declarations and contracts in
// include/reactflow.h).  Host side: argument checks, mechanism packing,
// workspace management and the launch sequence of one RHS evaluation / one
// SSP-RK3 step.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "reactflow.h"
#include "rf_ensemble.cuh"
#include "rf_adjoint.cuh"

using namespace rf;

// ----------------------------------------------------------------------------- errors

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return (void)cudaGetLastError(), fail(e_ == cudaErrorMemoryAllocation ? RF_ENOMEM : RF_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

#define LAUNCH_CHECK()                                                                             \
    do {                                                                                           \
        cudaError_t e_ = cudaGetLastError();                                                       \
        if (e_ != cudaSuccess)                                                                     \
            return fail(RF_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

extern "C" const char *rf_last_error(void) { return g_err.c_str(); }

// ----------------------------------------------------------------------------- objects

static constexpr int RF_MAX_DEVICES = 64;

struct rf_mech {
    MechDev d;
    int ns, nr;
    int npress;                      // pressure-dependent reactions
    int slot[RF_MAX_DEVICES];        // constant-memory slot per device, -1 if not uploaded
};

// Owners of the constant-memory mechanism slots of every device.
static std::mutex g_slot_mutex;
static const rf_mech *g_slot_owner[RF_MAX_DEVICES][MECH_SLOTS];

static bool g_exp_tab_done[RF_MAX_DEVICES];

// Tables of the FP64 exponential (2^(j/256) and 2^(-j/256), j = 0..255) and
// logarithm, rounded from extended precision, on device dev; the caller holds
// g_slot_mutex.
static int upload_exp_table(int dev) {
    if (g_exp_tab_done[dev]) return RF_OK;
    double tab[512];
    for (int j = 0; j < 256; ++j) {
        tab[j] = (double)std::exp2l((long double)j / 256.0L);
        tab[256 + j] = (double)std::exp2l(-(long double)j / 256.0L);
    }
    CUDA_TRY(cudaMemcpyToSymbol(g_exp_tab, tab, sizeof(tab)));
    // logarithm table: 1/F, ln F split into high and low parts, F = 1 + j/64
    double ltab[65 * 3];
    for (int j = 0; j <= 64; ++j) {
        const long double F = 1.0L + (long double)j / 64.0L;
        const long double lf = std::log(F);
        ltab[3 * j] = (double)(1.0L / F);
        ltab[3 * j + 1] = (double)lf;
        ltab[3 * j + 2] = (double)(lf - (long double)ltab[3 * j + 1]);
    }
    CUDA_TRY(cudaMemcpyToSymbol(g_log_tab, ltab, sizeof(ltab)));
    g_exp_tab_done[dev] = true;
    return RF_OK;
}

// Constant-memory slot of m on the current device, uploading it (and the
// exponential table) on first use.
static int mech_slot(const rf_mech *mc, int *out) {
    rf_mech *m = const_cast<rf_mech *>(mc);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= RF_MAX_DEVICES) return fail(RF_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    if (int rc = upload_exp_table(dev)) return rc;
    if (m->slot[dev] >= 0) {
        *out = m->slot[dev];
        return RF_OK;
    }
    for (int k = 0; k < MECH_SLOTS; ++k) {
        if (g_slot_owner[dev][k]) continue;
        CUDA_TRY(cudaMemcpyToSymbol(c_mech, &m->d, sizeof(MechDev), k * sizeof(MechDev)));
        g_slot_owner[dev][k] = m;
        m->slot[dev] = k;
        *out = k;
        return RF_OK;
    }
    return fail(RF_EINVAL, "at most %d mechanisms can be in use on one device (free unused ones)", MECH_SLOTS);
}

enum { PROF_CELL = 0, PROF_SWEEP_X = 1, PROF_SWEEP_Y = 2, PROF_SWEEP_Z = 3, PROF_OTHER = 4, RF_NPROF = 5 };

struct rf_ctx {
    const rf_mech *mech;
    int mslot = 0;                           // constant-memory slot of the mechanism
    rf_grid_desc g;
    int precision;
    uint32_t flags;
    long long n;
    int ns, nv, nq;
    size_t rsize;
    void *Q = nullptr, *rhs = nullptr;
    float *U32 = nullptr;
    double *U1 = nullptr, *U2 = nullptr;
    double *clock = nullptr;                 // t, dt, cfl, dt_fixed
    unsigned long long *rates = nullptr;
    int *status = nullptr;
    long long *bad_cell = nullptr;
    double *diag = nullptr;                  // partial sums + folded result
    int diag_blocks = 0;
    int newton_maxit = 30;
    int x_block = 256;                       // x sweep threads per block
    int walk_block = 128, walk_seg = 16;     // y / z sweeps (FP64 path)
    int walk_seg_staged = 32;                // y / z sweeps (staged FP32-bulk path): cells per segment
    size_t bytes = 0;
    // adjoint workspace (FP64 contexts), allocated on first use
    double *adj = nullptr;                   // Qbar [nq n], zero [nv n], R [nv n], lamS [nv n], Ub1, Ub2, Ln [nv n], T0, T1, T2 [n]
    // host-buffer step: device copies of U and T, a copy stream and its chunk events
    double *hU = nullptr, *hT = nullptr;
    cudaStream_t copy = nullptr;
    // host-buffer step: [0, 8) chunk copies in, [8] queued work before them, [9] the last
    // stage's cell state (T final), [10] T copied out
    cudaEvent_t hev[11] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // host-buffer step, copy out: a second copy stream (so copies out of one step and
    // in of the next run in both directions at once), [0, 8) chunk copies out done,
    // [8] the last stage done; out_pending: a step's copies out may still be in flight
    cudaStream_t copy_out = nullptr;
    cudaEvent_t oev[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int out_pending = 0;
    // optional per-kernel timing: CUDA events recorded on the launching stream
    int profile = 0;
    std::vector<cudaEvent_t> ev[RF_NPROF][2];
    // characteristic boundaries of the axes whose bc is RF_BC_NSCBC (rf_set_nscbc) and a
    // counter of their changes (ensembles re-capture their graphs when it moves)
    NscbcAxis nscbc[3];
    long long nscbc_version = 0;
    // mapped grids (RF_MAPPED): face area vectors, cell metric, volume, 1/volume (bulk
    // type) and cell centres (FP64), filled by rf_set_nodes
    int nodes_set = 0;
    void *geo = nullptr;
    void *gS[3] = {nullptr, nullptr, nullptr};
    void *gM = nullptr, *giV = nullptr;
    double *gV = nullptr, *gC = nullptr;
};

// record a start event before and a stop event after one launch of class k
struct ProfScope {
    rf_ctx *c;
    int k;
    cudaStream_t s;
    ProfScope(rf_ctx *c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
        if (c->profile) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            cudaEventRecord(e, s);
            c->ev[k][0].push_back(e);
        }
    }
    ~ProfScope() {
        if (c->profile) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            cudaEventRecord(e, s);
            c->ev[k][1].push_back(e);
        }
    }
};

static bool supported_ns(int ns) { return ns == 1 || ns == 2 || ns == 4 || ns == 9; }

extern "C" int rf_init_mechanism(const rf_mech_desc *d, rf_mech **out) {
    if (!d || !out) return fail(RF_EINVAL, "rf_init_mechanism: null argument");
    *out = nullptr;
    const int ns = d->n_species, nr = d->n_reactions;
    if (!supported_ns(ns)) return fail(RF_EINVAL, "rf_init_mechanism: n_species=%d not supported (1, 2, 4 or 9)", ns);
    if (nr < 0 || nr > NRMAX) return fail(RF_EINVAL, "rf_init_mechanism: n_reactions=%d outside [0, %d]", nr, NRMAX);
    if (!d->W || !d->nasa_low || !d->nasa_high || !d->T_mid || !d->mu_ref || !d->mu_exp || !d->D_ref)
        return fail(RF_EINVAL, "rf_init_mechanism: null species array");
    if (nr > 0 && (!d->A || !d->b || !d->Theta || !d->nu_f || !d->nu_r || !d->reversible))
        return fail(RF_EINVAL, "rf_init_mechanism: null reaction array");
    rf_mech *m = new rf_mech();
    std::memset(&m->d, 0, sizeof(MechDev));
    for (int k = 0; k < RF_MAX_DEVICES; ++k) m->slot[k] = -1;
    MechDev &M = m->d;
    M.ns = ns;
    M.nr = nr;
    m->ns = ns;
    m->nr = nr;
    M.Tmid = d->T_mid[0];
    bool same = true;
    for (int s = 0; s < ns; ++s) {
        if (d->T_mid[s] != M.Tmid) {
            delete m;
            return fail(RF_EINVAL, "rf_init_mechanism: species %d has T_mid %g != %g (one T_mid required)", s, d->T_mid[s], M.Tmid);
        }
        if (!(d->W[s] > 0.0)) {
            delete m;
            return fail(RF_EINVAL, "rf_init_mechanism: W[%d] = %g must be > 0", s, d->W[s]);
        }
        for (int k = 0; k < 7; ++k) same = same && d->nasa_low[s * 7 + k] == d->nasa_high[s * 7 + k];
    }
    M.two_ranges = same ? 0 : 1;
    for (int s = 0; s < ns; ++s) {
        M.W[s] = d->W[s];
        M.invW[s] = 1.0 / d->W[s];
        M.RW[s] = RU / d->W[s];
        for (int r = 0; r < 2; ++r) {
            const double *a = (r == 0 ? d->nasa_low : d->nasa_high) + s * 7;
            for (int k = 0; k < 5; ++k) M.cpc[r][s][k] = a[k];
            M.ec[r][s][0] = a[0];
            M.ec[r][s][1] = a[1] / 2.0;
            M.ec[r][s][2] = a[2] / 3.0;
            M.ec[r][s][3] = a[3] / 4.0;
            M.ec[r][s][4] = a[4] / 5.0;
            M.ec[r][s][5] = a[5];
            // e_s = h_s - (R/W_s) T: the linear coefficient takes the -R/W_s
            for (int k = 0; k < 6; ++k) M.ecR[r][s][k] = M.ec[r][s][k] * M.RW[s];
            M.ecR[r][s][0] = (M.ec[r][s][0] - 1.0) * M.RW[s];
            // ln G_s = g_s/RT + ln(R T / p_atm): the constant and the ln T coefficient absorb the second term
            M.gc[r][s][0] = a[0] - a[6] + std::log(RU / PATM);
            M.gc[r][s][1] = -a[1] / 2.0;
            M.gc[r][s][2] = -a[2] / 6.0;
            M.gc[r][s][3] = -a[3] / 12.0;
            M.gc[r][s][4] = -a[4] / 20.0;
            M.gc[r][s][5] = a[5];
            M.gc[r][s][6] = 1.0 - a[0];
            M.gc0w[r][s] = M.gc[r][s][0] - std::log(d->W[s]);
            for (int k = 0; k < 5; ++k) M.cpcf[r][s][k] = (float)a[k];
            for (int k = 0; k < 6; ++k) M.ecf[r][s][k] = (float)M.ec[r][s][k];
        }
        M.mu_ref[s] = d->mu_ref[s];
        M.mu_exp[s] = d->mu_exp[s];
        M.hl_mu_ref[s] = 0.5 * std::log(d->mu_ref[s]);
        M.h_mu_exp[s] = 0.5 * d->mu_exp[s];
        M.eucken[s] = 1.25 * RU / d->W[s];
        M.Wf[s] = (float)M.W[s];
        M.invWf[s] = (float)M.invW[s];
        M.RWf[s] = (float)M.RW[s];
        M.mu_reff[s] = (float)M.mu_ref[s];
        M.mu_expf[s] = (float)M.mu_exp[s];
        M.euckenf[s] = (float)M.eucken[s];
        for (int j = 0; j < ns; ++j) {
            const double D = d->D_ref[s * ns + j];
            if (s != j && !(D > 0.0)) {
                delete m;
                return fail(RF_EINVAL, "rf_init_mechanism: D_ref[%d][%d] = %g must be > 0", s, j, D);
            }
            M.invDref[s][j] = s == j ? 0.0 : 1.0 / D;
            M.wc[s][j] = std::pow(d->W[j] / d->W[s], 0.25);
            M.wd[s][j] = 1.0 / std::sqrt(8.0 * (1.0 + d->W[s] / d->W[j]));
            M.invDreff[s][j] = (float)M.invDref[s][j];
            M.wcf[s][j] = (float)M.wc[s][j];
            M.wdf[s][j] = (float)M.wd[s][j];
        }
    }
    for (int j = 0; j < nr; ++j) {
        if (!(d->A[j] > 0.0)) {
            delete m;
            return fail(RF_EINVAL, "rf_init_mechanism: A[%d] = %g must be > 0", j, d->A[j]);
        }
        M.A[j] = d->A[j];
        M.lnA[j] = std::log(d->A[j]);
        M.b[j] = d->b[j];
        M.Theta[j] = d->Theta[j];
        M.lnAf[j] = (float)M.lnA[j];
        M.bf[j] = (float)M.b[j];
        M.Thetaf[j] = (float)M.Theta[j];
        M.rev[j] = d->reversible[j] ? 1 : 0;
        int nrc = 0, npd = 0, nnet = 0, dsum = 0;
        for (int s = 0; s < ns; ++s) {
            const int f = d->nu_f[j * ns + s], r = d->nu_r[j * ns + s];
            if (f < 0 || r < 0) {
                delete m;
                return fail(RF_EINVAL, "rf_init_mechanism: negative stoichiometric coefficient in reaction %d", j);
            }
            for (int q = 0; q < f; ++q) {
                if (nrc >= 3) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: reaction %d has more than 3 reactant molecules", j); }
                M.reac[j][nrc++] = (int8_t)s;
            }
            for (int q = 0; q < r; ++q) {
                if (npd >= 3) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: reaction %d has more than 3 product molecules", j); }
                M.prod[j][npd++] = (int8_t)s;
            }
            if (r - f != 0) {
                M.net_sp[j][nnet] = (int8_t)s;
                M.net_nu[j][nnet] = (int8_t)(r - f);
                ++nnet;
                dsum += r - f;
            }
        }
        M.n_reac[j] = (int8_t)nrc;
        {
            double kap = 1.0;
            for (int k = 0; k < nrc; ++k) kap /= d->W[M.reac[j][k]];
            M.kapf[j] = (float)kap;
        }
        M.n_prod[j] = (int8_t)npd;
        M.n_net[j] = (int8_t)nnet;
        M.dnu_sum[j] = (int8_t)dsum;
        int nf = 0;
        for (int k = 0; k < npd; ++k) M.revf[j][nf++] = M.prod[j][k];
        for (int k = 0; k < nrc; ++k) M.revf[j][nf++] = (int8_t)(M.reac[j][k] + 16);
        M.n_revf[j] = (int8_t)nf;
        for (int k = 0; k < nrc; ++k) {
            const int sp = M.reac[j][k];
            M.dnu_reac[j][k] = (int8_t)(d->nu_r[j * ns + sp] - d->nu_f[j * ns + sp]);
        }
        for (int k = 0; k < npd; ++k) {
            const int sp = M.prod[j][k];
            M.dnu_prod[j][k] = (int8_t)(d->nu_r[j * ns + sp] - d->nu_f[j * ns + sp]);
        }
        M.pslot[j] = -1;
        const int kind = d->rxn_type ? d->rxn_type[j] : 0;
        if (kind < 0 || kind > 3) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: rxn_type[%d] = %d unknown", j, kind); }
        if (kind == 0) continue;
        if (m->npress >= NPMAX) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: more than %d pressure-dependent reactions", NPMAX); }
        if (!d->efficiency || (kind >= 2 && (!d->A0 || !d->b0 || !d->Theta0)) || (kind == 3 && !d->troe)) {
            delete m;
            return fail(RF_EINVAL, "rf_init_mechanism: reaction %d of type %d lacks its efficiency / fall-off arrays", j, kind);
        }
        const int p = m->npress++;
        M.ptype[j] = (int8_t)kind;
        M.pslot[j] = (int8_t)p;
        for (int s2 = 0; s2 < ns; ++s2) {
            const double e = d->efficiency[j * ns + s2];
            if (!(e >= 0.0)) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: efficiency[%d][%d] = %g must be >= 0", j, s2, e); }
            M.eff[p][s2] = e;
            M.efff[p][s2] = (float)e;
        }
        if (kind >= 2) {
            if (!(d->A0[j] > 0.0)) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: A0[%d] = %g must be > 0", j, d->A0[j]); }
            M.lnA0[p] = std::log(d->A0[j]);
            M.b0[p] = d->b0[j];
            M.Theta0[p] = d->Theta0[j];
            M.lnA0f[p] = (float)M.lnA0[p];
            M.b0f[p] = (float)M.b0[p];
            M.Theta0f[p] = (float)M.Theta0[p];
        }
        if (kind == 3) {
            const double *tr = d->troe + 4 * j;
            if (!(tr[1] > 0.0 && tr[2] > 0.0)) { delete m; return fail(RF_EINVAL, "rf_init_mechanism: Troe T***, T* of reaction %d must be > 0", j); }
            for (int k = 0; k < 4; ++k) {
                M.troe[p][k] = tr[k];
                M.troef[p][k] = (float)tr[k];
            }
        }
    }
    M.npress = m->npress;
    // shape classes of the mixed path's rate-of-progress pass, and the species-major
    // net coefficient lists (reactions ascending)
    {
        int nc[5] = {0, 0, 0, 0, 0};
        auto cls = [&](int j) {
            const int a = M.n_reac[j], b = M.n_prod[j];
            if (!M.rev[j] || M.ptype[j] || a < 1 || a > 2 || b < 1 || b > 2) return 4;
            return (a - 1) * 2 + (b - 1);
        };
        for (int j = 0; j < nr; ++j) ++nc[cls(j)];
        M.cls_start[0] = 0;
        for (int c = 0; c < 5; ++c) M.cls_start[c + 1] = (int8_t)(M.cls_start[c] + nc[c]);
        int fill[5];
        for (int c = 0; c < 5; ++c) fill[c] = M.cls_start[c];
        for (int j = 0; j < nr; ++j) M.cls_rx[fill[cls(j)]++] = (int8_t)j;
        int e = 0;
        for (int s2 = 0; s2 < ns; ++s2) {
            M.sp_start[s2] = (int16_t)e;
            for (int j = 0; j < nr; ++j)
                for (int k = 0; k < M.n_net[j]; ++k)
                    if (M.net_sp[j][k] == s2) {
                        M.sp_rx[e] = (int8_t)j;
                        M.sp_nu[e] = M.net_nu[j][k];
                        ++e;
                    }
        }
        M.sp_start[ns] = (int16_t)e;
    }
    *out = m;
    return RF_OK;
}

extern "C" void rf_free_mechanism(rf_mech *m) {
    if (!m) return;
    {
        std::lock_guard<std::mutex> lock(g_slot_mutex);
        for (int dev = 0; dev < RF_MAX_DEVICES; ++dev)
            if (m->slot[dev] >= 0 && g_slot_owner[dev][m->slot[dev]] == m) g_slot_owner[dev][m->slot[dev]] = nullptr;
    }
    delete m;
}

static void free_ctx_buffers(rf_ctx *c) {
    void *ptrs[] = {c->Q, c->rhs, c->U32, c->U1, c->U2, c->clock, c->rates, c->status, c->bad_cell, c->diag, c->adj,
                    c->hU, c->hT, c->geo};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->hev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->oev)
        if (e) cudaEventDestroy(e);
    if (c->copy) cudaStreamDestroy(c->copy);
    if (c->copy_out) cudaStreamDestroy(c->copy_out);
}

static void clear_profile(rf_ctx *c) {
    for (int k = 0; k < RF_NPROF; ++k)
        for (int q = 0; q < 2; ++q) {
            for (cudaEvent_t e : c->ev[k][q]) cudaEventDestroy(e);
            c->ev[k][q].clear();
        }
}

extern "C" void rf_free_ctx(rf_ctx *c) {
    if (!c) return;
    clear_profile(c);
    free_ctx_buffers(c);
    delete c;
}

extern "C" size_t rf_ctx_workspace_bytes(const rf_ctx *c) { return c ? c->bytes : 0; }

static int prepare_ctx(rf_ctx *c);

// mapped-grid workspace: face area vectors of the three axes, cell metric, volume and
// its reciprocal in the bulk type, cell centres and a bad-cell counter in FP64 / u64
static size_t geo_faces(const rf_grid_desc &g, int a) {
    return a == 0 ? (size_t)(g.nx + 1) * g.ny * g.nz : (a == 1 ? (size_t)g.nx * (g.ny + 1) * g.nz : (size_t)g.nx * g.ny * (g.nz + 1));
}
static size_t geo_bytes(const rf_grid_desc &g, size_t rsize) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t r = 3 * (geo_faces(g, 0) + geo_faces(g, 1) + geo_faces(g, 2)) + 10 * n;
    return ((r * rsize + 15) / 16) * 16 + 4 * n * sizeof(double) + 16;
}
static void geo_layout(rf_ctx *c) {
    const size_t n = (size_t)c->n;
    char *p = (char *)c->geo;
    for (int a = 0; a < 3; ++a) {
        c->gS[a] = p;
        p += 3 * geo_faces(c->g, a) * c->rsize;
    }
    c->gM = p;
    p += 9 * n * c->rsize;
    c->giV = p;
    p += n * c->rsize;
    p = (char *)c->geo + ((size_t)(p - (char *)c->geo + 15) / 16) * 16;
    c->gV = (double *)p;
    c->gC = c->gV + n;                         // then 3n centres and the bad-cell counter
}

extern "C" int rf_create_ctx(const rf_mech *m, const rf_grid_desc *g, int precision, uint32_t flags, rf_ctx **out) {
    if (!m || !g || !out) return fail(RF_EINVAL, "rf_create_ctx: null argument");
    *out = nullptr;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(RF_EINVAL, "rf_create_ctx: grid %dx%dx%d has an empty axis", g->nx, g->ny, g->nz);
    if (g->nx > 1024) return fail(RF_EINVAL, "rf_create_ctx: nx = %d exceeds 1024", g->nx);
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return fail(RF_EINVAL, "rf_create_ctx: grid spacing must be > 0");
    for (int a = 0; a < 3; ++a) {
        if (g->bc[a] != RF_BC_PERIODIC && g->bc[a] != RF_BC_EXTRAPOLATE && g->bc[a] != RF_BC_NSCBC)
            return fail(RF_EINVAL, "rf_create_ctx: bc[%d] = %d unknown", a, g->bc[a]);
        const int na = a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
        if (g->bc[a] == RF_BC_NSCBC && na < 3) return fail(RF_EINVAL, "rf_create_ctx: NSCBC axis %d has %d cells (needs >= 3)", a, na);
    }
    if (precision != RF_FP64 && precision != RF_MIXED) return fail(RF_EINVAL, "rf_create_ctx: precision %d unknown", precision);
    if (flags & ~(uint32_t)RF_FLAGS_ALL) return fail(RF_EINVAL, "rf_create_ctx: unknown flag bits 0x%x", flags & ~(uint32_t)RF_FLAGS_ALL);
    if (flags & RF_CHARWISE) {
        if (flags & RF_MAPPED) return fail(RF_EINVAL, "rf_create_ctx: RF_CHARWISE is built for Cartesian grids, not RF_MAPPED ones");
        for (int a = 0; a < 3; ++a)
            if (g->bc[a] == RF_BC_NSCBC)
                return fail(RF_EINVAL, "rf_create_ctx: RF_CHARWISE with an NSCBC axis (%d) is not built", a);
    }
    int mslot = 0;
    {
        int rc = mech_slot(m, &mslot);
        if (rc) return rc;
    }
    rf_ctx *c = new rf_ctx();
    c->mech = m;
    c->mslot = mslot;
    c->g = *g;
    c->precision = precision;
    c->flags = flags;
    c->n = (long long)g->nx * g->ny * g->nz;
    c->ns = m->ns;
    c->nv = m->ns + 4;
    c->nq = Q_X0 + 3 * m->ns;
    c->rsize = precision == RF_FP64 ? sizeof(double) : sizeof(float);
    // ell = 0: the kernel takes the domain length along the axis (n h; n / (|S| / V) of
    // the boundary cell on a mapped grid)
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 2; ++e) c->nscbc[a].s[e] = NscbcSide{101325.0, 0.25, 1.0, 1.0, 1.0, 1.0, 0.0, nullptr};
    const size_t n = (size_t)c->n;
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {&c->Q, n * c->nq * c->rsize},
        {&c->rhs, n * c->nv * c->rsize},
        {(void **)&c->U32, precision == RF_MIXED ? n * c->nv * sizeof(float) : 0},
        {(void **)&c->U1, n * c->nv * sizeof(double)},
        {(void **)&c->U2, n * c->nv * sizeof(double)},
        {(void **)&c->clock, 8 * sizeof(double)},
        {(void **)&c->rates, 4 * sizeof(unsigned long long)},
        {(void **)&c->status, sizeof(int) * 2},
        {(void **)&c->bad_cell, sizeof(long long)},
        {&c->geo, (flags & RF_MAPPED) ? geo_bytes(*g, c->rsize) : 0},
    };
    for (auto &a : allocs) {
        if (!a.bytes) continue;
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            free_ctx_buffers(c);
            delete c;
            return fail(RF_ENOMEM, "rf_create_ctx: cudaMalloc(%zu) failed: %s", a.bytes, cudaGetErrorString(e));
        }
        c->bytes += a.bytes;
    }
    c->diag_blocks = (int)((c->n + 63) / 64);
    cudaError_t e = cudaMalloc((void **)&c->diag, ((size_t)c->diag_blocks + 1) * (c->nv + 2) * sizeof(double));
    if (e != cudaSuccess) {
        free_ctx_buffers(c);
        delete c;
        return fail(RF_ENOMEM, "rf_create_ctx: diagnostics buffer: %s", cudaGetErrorString(e));
    }
    if (c->geo) geo_layout(c);
    cudaMemset(c->status, 0, sizeof(int) * 2);
    cudaMemset(c->bad_cell, 0xff, sizeof(long long));
    cudaMemset(c->clock, 0, 8 * sizeof(double));
    cudaMemset(c->rates, 0, 4 * sizeof(unsigned long long));
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_ctx_buffers(c);
        delete c;
        return fail(RF_ECUDA, "rf_create_ctx: %s", cudaGetErrorString(e));
    }
    if (int rc = prepare_ctx(c)) {
        free_ctx_buffers(c);
        delete c;
        return rc;
    }
    *out = c;
    return RF_OK;
}

// ----------------------------------------------------------------------------- launch sequence

static Member base_member(rf_ctx *c) {
    Member m;
    std::memset(&m, 0, sizeof m);
    m.nx = c->g.nx;
    m.ny = c->g.ny;
    m.nz = c->g.nz;
    for (int a = 0; a < 3; ++a) m.bc[a] = c->g.bc[a];
    m.h[0] = c->g.dx;
    m.h[1] = c->g.dy;
    m.h[2] = c->g.dz;
    for (int a = 0; a < 3; ++a) m.invh[a] = 1.0 / m.h[a];
    for (int a = 0; a < 3; ++a) m.weps[a] = m.h[a] * m.h[a] / 3.0;
    m.n = c->n;
    m.Q = c->Q;
    m.rhs = c->rhs;
    m.U32 = c->U32;
    m.clock = c->clock;
    m.rates = c->rates;
    m.status = c->status;
    m.bad_cell = c->bad_cell;
    m.flags = (int)c->flags;
    m.c_lo = 0;
    m.c_hi = c->n;
    if (c->flags & RF_MAPPED) {
        m.mapped = 1;
        for (int a = 0; a < 3; ++a) m.gS[a] = c->gS[a];
        m.gM = c->gM;
        m.gV = c->gV;
        m.giV = c->giV;
        m.gC = c->gC;
    }
    return m;
}

static void set_laser(Member &m, const rf_laser *L) {
    if (L && L->E != 0.0 && L->sigma_r > 0.0 && L->sigma_t > 0.0) {
        m.laser_on = 1;
        m.las[0] = L->E;
        m.las[1] = L->x0;
        m.las[2] = L->y0;
        m.las[3] = L->z0;
        m.las[4] = L->sigma_r;
        m.las[5] = L->t0;
        m.las[6] = L->sigma_t;
        // the time-independent factors of the source, once on the host
        const double two_pi = 6.283185307179586, sr = L->sigma_r, st = L->sigma_t;
        m.las_k[0] = m.nz == 1 ? L->E / (two_pi * std::sqrt(two_pi) * sr * sr * st)
                               : L->E / (two_pi * two_pi * sr * sr * sr * st);
        m.las_k[1] = -0.5 / (sr * sr);
        m.las_k[2] = 1.0 / st;
        for (int d = 0; d < 3; ++d) m.las_c0[d] = std::fma(0.5, m.h[d], -m.las[1 + d]);
    }
}

template <typename R, int NS>
struct Path {
    using UT = typename std::conditional<sizeof(R) == 4, float, double>::type;

    // kernel attributes, set once per context before any launch (or capture)
    static int prepare(rf_ctx *c) {
        CUDA_TRY(cudaFuncSetAttribute(cell_state_kernel<R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)cell_state_smem_max<R, NS>(128, c->mech->nr)));
        if constexpr (sizeof(R) == 4) {
            const int sm = (int)walk_smem<R, NS>();
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 1, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 1, MODE_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 1, MODE_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 2, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 2, MODE_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            CUDA_TRY(cudaFuncSetAttribute(sweep_walk_staged_kernel<NS, 2, MODE_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            const int sx = (int)XTile<NS>::SMEM;
            CUDA_TRY(cudaFuncSetAttribute(sweep_x_staged_kernel<NS, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx));
            CUDA_TRY(cudaFuncSetAttribute(sweep_x_staged_kernel<NS, MODE_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx));
            CUDA_TRY(cudaFuncSetAttribute(sweep_x_staged_kernel<NS, MODE_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx));
        }
        return RF_OK;
    }

    static int cell_state(rf_ctx *c, const Member &m, cudaStream_t s) {
        const int B = 128;
        const long long nb = (m.c_hi - m.c_lo + B - 1) / B;
        if (nb <= 0) return RF_OK;
        const size_t smem = cell_state_smem<R, NS>(B, m.want_rates != 0, c->mech->nr);
        ProfScope ps(c, PROF_CELL, s);
        cell_state_kernel<R, NS><<<(unsigned)nb, B, smem, s>>>(c->mslot, m, c->newton_maxit);
        LAUNCH_CHECK();
        return RF_OK;
    }

    // characteristic boundary terms of every NSCBC axis, after the cell state has
    // filled the RHS accumulator and before the sweeps add to it
    template <int DIR, int SCHEME>
    static void nscbc_axis(rf_ctx *c, const Member &m, cudaStream_t s) {
        const int nn[3] = {c->g.nx, c->g.ny, c->g.nz};
        const long long plane = (long long)nn[DIR == 0 ? 1 : 0] * nn[DIR == 2 ? 1 : 2];
        const unsigned blocks = (unsigned)((2 * plane + 127) / 128);
        if (c->flags & RF_MAPPED)
            nscbc_kernel<R, UT, NS, DIR, SCHEME, 1><<<blocks, 128, 0, s>>>(c->mslot, m, c->nscbc[DIR]);
        else
            nscbc_kernel<R, UT, NS, DIR, SCHEME, 0><<<blocks, 128, 0, s>>>(c->mslot, m, c->nscbc[DIR]);
    }

    static int nscbc(rf_ctx *c, const Member &m, cudaStream_t s) {
        if (m.flags & F_NO_INVISCID) return RF_OK;
        const bool teno = (c->flags & RF_TENO6) != 0;
        for (int d = 0; d < 3; ++d) {
            if (c->g.bc[d] != RF_BC_NSCBC) continue;
            ProfScope ps(c, PROF_OTHER, s);
            if (d == 0) teno ? nscbc_axis<0, 1>(c, m, s) : nscbc_axis<0, 0>(c, m, s);
            else if (d == 1) teno ? nscbc_axis<1, 1>(c, m, s) : nscbc_axis<1, 0>(c, m, s);
            else teno ? nscbc_axis<2, 1>(c, m, s) : nscbc_axis<2, 0>(c, m, s);
            LAUNCH_CHECK();
        }
        return RF_OK;
    }

    // TENO6 sweeps: thread per face from global memory (six-cell stencils), both precisions
    template <int MODE>
    static int sweep_teno(rf_ctx *c, const Member &m, int dir, cudaStream_t s) {
        return sweep_global<MODE, 1, 0>(c, m, dir, s);
    }

    // global-memory sweeps (thread per face) of scheme SCHEME on a Cartesian (GEOM 0) or
    // mapped (GEOM 1) grid, both precisions
    template <int MODE, int SCHEME, int GEOM>
    static int sweep_global(rf_ctx *c, const Member &m, int dir, cudaStream_t s) {
        constexpr int NV = NS + 4;
        // FP32 sweeps in register-capped kernels of 128-thread blocks, CAP blocks per SM:
        // characteristic-wise 3 (168 registers, 80 / 112 bytes of spills), mapped 4
        // (128, up to 44 bytes), TENO6 5 (96, 52 bytes)
        constexpr int CAP = sizeof(R) != 4 ? 0 : (SCHEME >= 2 ? 3 : (GEOM ? 4 : (SCHEME == 1 ? 5 : 0)));
        if (dir == 0) {
            const int nx = c->g.nx;
            const int xb = CAP ? std::min(c->x_block, 128) : c->x_block;
            int W, rpb;
            if (nx <= xb) {
                W = nx;
                rpb = std::max(1, std::min(xb / nx, 320 / (nx + 2)));
            } else {
                W = xb;
                rpb = 1;
            }
            const int threads = ((W * rpb + 31) / 32) * 32;
            const int nrows = c->g.ny * c->g.nz;
            const int blocks = (nrows + rpb - 1) / rpb;
            const size_t smem = (size_t)NV * rpb * (W + 2) * sizeof(R);
            ProfScope ps(c, PROF_SWEEP_X, s);
            if constexpr (CAP > 0)
                sweep_x_capped_kernel<UT, NS, MODE, SCHEME, GEOM, CAP><<<blocks, threads, smem, s>>>(c->mslot, m, W, rpb);
            else
                sweep_x_kernel<R, UT, NS, MODE, SCHEME, GEOM><<<blocks, threads, smem, s>>>(c->mslot, m, W, rpb);
        } else {
            const int nd = dir == 1 ? c->g.ny : c->g.nz;
            const long long lines = (long long)c->g.nx * (dir == 1 ? c->g.nz : c->g.ny);
            dim3 grid((unsigned)((lines + c->walk_block - 1) / c->walk_block), (unsigned)((nd + c->walk_seg - 1) / c->walk_seg));
            ProfScope ps(c, dir == 1 ? PROF_SWEEP_Y : PROF_SWEEP_Z, s);
            if constexpr (CAP > 0) {
                if (dir == 1)
                    sweep_walk_capped_kernel<UT, NS, 1, MODE, SCHEME, GEOM, CAP><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
                else
                    sweep_walk_capped_kernel<UT, NS, 2, MODE, SCHEME, GEOM, CAP><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
            } else if (dir == 1)
                sweep_walk_kernel<R, UT, NS, 1, MODE, SCHEME, GEOM><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
            else
                sweep_walk_kernel<R, UT, NS, 2, MODE, SCHEME, GEOM><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
        }
        LAUNCH_CHECK();
        return RF_OK;
    }

    template <int MODE>
    static int sweep(rf_ctx *c, const Member &m, int dir, cudaStream_t s) {
        constexpr int NV = NS + 4;
        if (c->flags & RF_MAPPED)
            return (c->flags & RF_TENO6) ? sweep_global<MODE, 1, 1>(c, m, dir, s) : sweep_global<MODE, 0, 1>(c, m, dir, s);
        if (c->flags & RF_CHARWISE)
            return (c->flags & RF_TENO6) ? sweep_global<MODE, 3, 0>(c, m, dir, s) : sweep_global<MODE, 2, 0>(c, m, dir, s);
        if (c->flags & RF_TENO6) return sweep_teno<MODE>(c, m, dir, s);
        if (dir == 0 && sizeof(R) == 4) {
            // staged x sweep: a row per warp, four rows per block
            const int nrows = c->g.ny * c->g.nz;
            const int blocks = (nrows + XTile<NS>::WARPS - 1) / XTile<NS>::WARPS;
            ProfScope ps(c, PROF_SWEEP_X, s);
            sweep_x_staged_kernel<NS, MODE><<<blocks, 128, XTile<NS>::SMEM, s>>>(c->mslot, m);
        } else if (dir == 0) {
            const int nx = c->g.nx;
            int W, rpb;
            if (nx <= c->x_block) {
                W = nx;
                // rows per block; the (W + 2)-slot row buffers stay within 320 slots
                // so that NV * rpb * (W + 2) * 8 bytes fits the 48 KB default
                rpb = std::max(1, std::min(c->x_block / nx, 320 / (nx + 2)));
            } else {
                W = c->x_block;
                rpb = 1;
            }
            const int threads = ((W * rpb + 31) / 32) * 32;
            const int nrows = c->g.ny * c->g.nz;
            const int blocks = (nrows + rpb - 1) / rpb;
            const size_t smem = (size_t)NV * rpb * (W + 2) * sizeof(R);
            ProfScope ps(c, PROF_SWEEP_X, s);
            sweep_x_kernel<R, UT, NS, MODE><<<blocks, threads, smem, s>>>(c->mslot, m, W, rpb);
        } else if (sizeof(R) == 4) {
            // staged walk: 32 x 4 line tiles, planes streamed through shared memory
            const int nd = dir == 1 ? c->g.ny : c->g.nz;
            const int no = dir == 1 ? c->g.nz : c->g.ny;
            const int seg = c->walk_seg_staged;
            dim3 grid((unsigned)walk_tiles<R, NS>(c->g.nx, no), (unsigned)((nd + seg - 1) / seg));
            const size_t smem = walk_smem<R, NS>();
            ProfScope ps(c, dir == 1 ? PROF_SWEEP_Y : PROF_SWEEP_Z, s);
            if (dir == 1)
                sweep_walk_staged_kernel<NS, 1, MODE><<<grid, 128, smem, s>>>(c->mslot, m, seg);
            else
                sweep_walk_staged_kernel<NS, 2, MODE><<<grid, 128, smem, s>>>(c->mslot, m, seg);
        } else {
            const int nd = dir == 1 ? c->g.ny : c->g.nz;
            const long long lines = (long long)c->g.nx * (dir == 1 ? c->g.nz : c->g.ny);
            dim3 grid((unsigned)((lines + c->walk_block - 1) / c->walk_block), (unsigned)((nd + c->walk_seg - 1) / c->walk_seg));
            ProfScope ps(c, dir == 1 ? PROF_SWEEP_Y : PROF_SWEEP_Z, s);
            if (dir == 1)
                sweep_walk_kernel<R, UT, NS, 1, MODE><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
            else
                sweep_walk_kernel<R, UT, NS, 2, MODE><<<grid, c->walk_block, 0, s>>>(c->mslot, m, c->walk_seg);
        }
        LAUNCH_CHECK();
        return RF_OK;
    }

    // all sweeps of one evaluation; the last active axis runs in mode MODE
    template <int MODE>
    static int sweeps(rf_ctx *c, const Member &m, cudaStream_t s) {
        const int n[3] = {c->g.nx, c->g.ny, c->g.nz};
        int last = -1;
        for (int d = 0; d < 3; ++d)
            if (n[d] > 1) last = d;
        if (last < 0) {
            ProfScope ps(c, PROF_OTHER, s);
            pointwise_final_kernel<R, NS, MODE><<<(unsigned)((c->n + 127) / 128), 128, 0, s>>>(m);
            LAUNCH_CHECK();
            return RF_OK;
        }
        // FP32-bulk RK stages: every sweep accumulates, then an elementwise FP64
        // Shu-Osher update (the same values as fusing it into the last sweep, whose
        // FP64 operations would otherwise hold the sweep's few warps per SM)
        const bool split = sizeof(R) == 4 && MODE == MODE_STAGE;
        for (int d = 0; d < 3; ++d) {
            if (n[d] <= 1) continue;
            int rc = (d == last && !split) ? sweep<MODE>(c, m, d, s) : sweep<MODE_ACCUM>(c, m, d, s);
            if (rc) return rc;
        }
        if (split) {
            ProfScope ps(c, PROF_OTHER, s);
            pointwise_final_kernel<R, NS, MODE><<<(unsigned)((c->n + 255) / 256), 256, 0, s>>>(m);
            LAUNCH_CHECK();
        }
        return RF_OK;
    }

    static int rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, double *dUdt, cudaStream_t s) {
        Member m = base_member(c);
        m.U = U;
        m.T = T;
        m.dUdt = dUdt;
        m.t_from_host = 1;
        m.t_host = t;
        set_laser(m, L);
        int rc = cell_state(c, m, s);
        if (rc) return rc;
        if ((rc = nscbc(c, m, s))) return rc;
        return sweeps<MODE_RHS>(c, m, s);
    }

    // chunks > 0: the first stage's cell state runs on cells [q n / chunks, (q + 1) n / chunks)
    // once chunk_ev[q] has completed (the host-buffer step streams the state in by chunks)
    // t_final_ev (if given) is recorded once the last stage's cell state has written T
    static int rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl, const rf_laser *L,
                       double *dt_dev, cudaStream_t s, int chunks = 0, const cudaEvent_t *chunk_ev = nullptr,
                       cudaEvent_t t_final_ev = nullptr) {
        // clock = (t, dt, cfl, dt_fixed)
        double hostclk[2] = {cfl, dt_fixed};
        CUDA_TRY(cudaMemcpyAsync(c->clock, t_dev, sizeof(double), cudaMemcpyDeviceToDevice, s));
        step_params_kernel<<<1, 1, 0, s>>>(c->clock, hostclk[0], hostclk[1], c->rates);
        LAUNCH_CHECK();
        Member m = base_member(c);
        m.T = T;
        m.Un = U;
        set_laser(m, L);
        const double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0}, cc[3] = {0.0, 1.0, 0.5};
        const double *in[3] = {U, c->U1, c->U2};
        double *outp[3] = {c->U1, c->U2, U};
        // a mapped grid's diffusive rate already carries max_e |grad xi_e|^2
        const double hmin = (c->flags & RF_MAPPED) ? 1.0
                                                   : std::min(c->g.nx > 1 ? c->g.dx : 1e300,
                                                              std::min(c->g.ny > 1 ? c->g.dy : 1e300, c->g.nz > 1 ? c->g.dz : 1e300));
        for (int k = 0; k < 3; ++k) {
            m.U = in[k];
            m.Uout = outp[k];
            m.stage_a = a[k];
            m.stage_b = b[k];
            m.stage_c = cc[k];
            m.want_rates = (k == 0 && !(dt_fixed > 0.0)) ? 1 : 0;
            int rc;
            if (k == 0 && chunks > 0) {
                for (int q = 0; q < chunks; ++q) {
                    Member mq = m;
                    mq.c_lo = c->n * q / chunks;
                    mq.c_hi = c->n * (q + 1) / chunks;
                    CUDA_TRY(cudaStreamWaitEvent(s, chunk_ev[q], 0));
                    if ((rc = cell_state(c, mq, s))) return rc;
                }
            } else if ((rc = cell_state(c, m, s))) {
                return rc;
            }
            if (k == 2 && t_final_ev) CUDA_TRY(cudaEventRecord(t_final_ev, s));
            if ((rc = nscbc(c, m, s))) return rc;
            if (k == 0) {
                dt_kernel<<<1, 1, 0, s>>>(c->clock, c->rates, hmin, !(c->flags & RF_NO_VISCOUS),
                                          !(c->flags & RF_NO_CHEMISTRY) && c->mech->nr > 0, m.laser_on && !(c->flags & RF_NO_LASER),
                                          m.las[5], m.las[6], dt_dev);
                LAUNCH_CHECK();
            }
            rc = sweeps<MODE_STAGE>(c, m, s);
            if (rc) return rc;
        }
        step_end_kernel<<<1, 1, 0, s>>>(c->clock, t_dev);
        LAUNCH_CHECK();
        return RF_OK;
    }

    static int init_state(rf_ctx *c, const double *prim, double *U, double *T, cudaStream_t s) {
        init_state_kernel<NS><<<(unsigned)((c->n + 127) / 128), 128, 0, s>>>(c->mslot, prim, U, T, c->n);
        LAUNCH_CHECK();
        return RF_OK;
    }

    static int diagnostics(rf_ctx *c, const double *U, double *T, rf_diag *out, cudaStream_t s) {
        Member m = base_member(c);
        m.U = U;
        m.T = T;
        const int B = 64;
        const size_t smem = (size_t)B * NS * 5 * sizeof(double);
        diag_kernel<NS><<<c->diag_blocks, B, smem, s>>>(c->mslot, m, c->diag, c->newton_maxit);
        LAUNCH_CHECK();
        const int nvals = NS + 6;
        double *res = c->diag + (size_t)c->diag_blocks * nvals;
        diag_fold_kernel<<<1, 32 * nvals, 0, s>>>(c->diag, c->diag_blocks, nvals, res);
        LAUNCH_CHECK();
        double host[32];
        CUDA_TRY(cudaMemcpyAsync(host, res, nvals * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        std::memset(out, 0, sizeof(rf_diag));
        out->nv = NS + 4;
        for (int v = 0; v < NS + 4; ++v) out->total[v] = host[v];
        out->heat_release = host[NS + 4];
        out->max_T = host[NS + 5];
        return RF_OK;
    }
};

#define DISPATCH(c, CALL)                                                            \
    do {                                                                             \
        if ((c)->precision == RF_FP64) {                                             \
            switch ((c)->ns) {                                                       \
                case 1: return Path<double, 1>::CALL;                                \
                case 2: return Path<double, 2>::CALL;                                \
                case 4: return Path<double, 4>::CALL;                                \
                case 9: return Path<double, 9>::CALL;                                \
            }                                                                        \
        } else {                                                                     \
            switch ((c)->ns) {                                                       \
                case 1: return Path<float, 1>::CALL;                                 \
                case 2: return Path<float, 2>::CALL;                                 \
                case 4: return Path<float, 4>::CALL;                                 \
                case 9: return Path<float, 9>::CALL;                                 \
            }                                                                        \
        }                                                                            \
        return fail(RF_EINVAL, "unsupported species count %d", (c)->ns);             \
    } while (0)

// Kernel attributes of a context's precision and species count (dynamic shared
// memory above the default 48 KB).
static int prepare_ctx(rf_ctx *c) { DISPATCH(c, prepare(c)); }

extern "C" int rf_init_state(rf_ctx *c, const double *prim, double *U, double *T, rf_stream s) {
    if (!c || !prim || !U || !T) return fail(RF_EINVAL, "rf_init_state: null argument");
    DISPATCH(c, init_state(c, prim, U, T, (cudaStream_t)s));
}

#define NODES_READY(c, where)                                                                     \
    do {                                                                                          \
        if (((c)->flags & RF_MAPPED) && !(c)->nodes_set)                                          \
            return fail(RF_EINVAL, "%s: mapped context without node coordinates (rf_set_nodes)", where); \
    } while (0)

extern "C" int rf_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, double *dUdt, rf_stream s) {
    if (!c || !U || !T || !dUdt) return fail(RF_EINVAL, "rf_rhs: null argument");
    NODES_READY(c, "rf_rhs");
    DISPATCH(c, rhs(c, U, T, t, L, dUdt, (cudaStream_t)s));
}

extern "C" int rf_rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl, const rf_laser *L,
                          double *dt_dev, rf_stream s) {
    if (!c || !U || !T || !t_dev) return fail(RF_EINVAL, "rf_rk_step: null argument");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(RF_EINVAL, "rf_rk_step: need dt_fixed > 0 or cfl > 0");
    NODES_READY(c, "rf_rk_step");
    DISPATCH(c, rk_step(c, U, T, t_dev, dt_fixed, cfl, L, dt_dev, (cudaStream_t)s));
}

static int rk_step_chunked(rf_ctx *c, double *t_dev, double dt_fixed, double cfl, const rf_laser *L, double *dt_dev,
                           cudaStream_t s, int chunks) {
    DISPATCH(c, rk_step(c, c->hU, c->hT, t_dev, dt_fixed, cfl, L, dt_dev, s, chunks, c->hev, c->hev[9]));
}

extern "C" int rf_rk_step_host(rf_ctx *c, const double *U_in, const double *T_in, double *U_out, double *T_out,
                               double *t_dev, double dt_fixed, double cfl, const rf_laser *L, double *dt_dev,
                               rf_stream s) {
    if (!c || !U_in || !T_in || !U_out || !t_dev) return fail(RF_EINVAL, "rf_rk_step_host: null argument");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(RF_EINVAL, "rf_rk_step_host: need dt_fixed > 0 or cfl > 0");
    NODES_READY(c, "rf_rk_step_host");
    const long long n = c->n;
    const int nv = c->nv;
    if (!c->hU) {
        CUDA_TRY(cudaMalloc((void **)&c->hU, (size_t)n * nv * sizeof(double)));
        CUDA_TRY(cudaMalloc((void **)&c->hT, (size_t)n * sizeof(double)));
        c->bytes += (size_t)n * (nv + 1) * sizeof(double);
    }
    if (!c->copy) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->hev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t &e : c->oev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    cudaStream_t st = (cudaStream_t)s;
    const int chunks = (int)std::min<long long>(8, n);
    // The copies in overwrite hU / hT.  The first call's follow the work already queued on
    // s; a later call's follow the previous step's last stage (its last read of hU / hT on
    // s) and, chunk by chunk, that step's copy out of the same chunk (the host buffers may
    // be the same, and hU is that copy's source), so that the copies in of this step run
    // beside the remaining copies out of the previous one
    if (c->out_pending) {
        CUDA_TRY(cudaStreamWaitEvent(c->copy, c->oev[8], 0));
    } else {
        CUDA_TRY(cudaEventRecord(c->hev[8], st));
        CUDA_TRY(cudaStreamWaitEvent(c->copy, c->hev[8], 0));
    }
    for (int q = 0; q < chunks; ++q) {
        const long long lo = n * q / chunks, hi = n * (q + 1) / chunks;
        if (c->out_pending) CUDA_TRY(cudaStreamWaitEvent(c->copy, c->oev[q], 0));
        for (int v = 0; v < nv; ++v)
            CUDA_TRY(cudaMemcpyAsync(c->hU + (size_t)v * n + lo, U_in + (size_t)v * n + lo, (size_t)(hi - lo) * sizeof(double),
                                     cudaMemcpyHostToDevice, c->copy));
        CUDA_TRY(cudaMemcpyAsync(c->hT + lo, T_in + lo, (size_t)(hi - lo) * sizeof(double), cudaMemcpyHostToDevice, c->copy));
        CUDA_TRY(cudaEventRecord(c->hev[q], c->copy));
    }
    if (int rc = rk_step_chunked(c, t_dev, dt_fixed, cfl, L, dt_dev, st, chunks)) return rc;
    // T is final after the last stage's cell state: its copy out overlaps that stage's
    // sweeps on the copy stream, and s waits for it, so completion of s covers it
    if (T_out) {
        CUDA_TRY(cudaStreamWaitEvent(c->copy, c->hev[9], 0));
        CUDA_TRY(cudaMemcpyAsync(T_out, c->hT, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->copy));
        CUDA_TRY(cudaEventRecord(c->hev[10], c->copy));
    }
    // U out by chunks on the second copy stream once the last stage is done; s waits for
    // the last chunk, so completion of s covers the copies
    CUDA_TRY(cudaEventRecord(c->oev[8], st));
    CUDA_TRY(cudaStreamWaitEvent(c->copy_out, c->oev[8], 0));
    for (int q = 0; q < chunks; ++q) {
        const long long lo = n * q / chunks, hi = n * (q + 1) / chunks;
        for (int v = 0; v < nv; ++v)
            CUDA_TRY(cudaMemcpyAsync(U_out + (size_t)v * n + lo, c->hU + (size_t)v * n + lo, (size_t)(hi - lo) * sizeof(double),
                                     cudaMemcpyDeviceToHost, c->copy_out));
        CUDA_TRY(cudaEventRecord(c->oev[q], c->copy_out));
    }
    c->out_pending = 1;
    CUDA_TRY(cudaStreamWaitEvent(st, c->oev[chunks - 1], 0));
    if (T_out) CUDA_TRY(cudaStreamWaitEvent(st, c->hev[10], 0));
    return RF_OK;
}

extern "C" int rf_diagnostics(rf_ctx *c, const double *U, double *T, rf_diag *out, rf_stream s) {
    if (!c || !U || !T || !out) return fail(RF_EINVAL, "rf_diagnostics: null argument");
    if (c->nv + 2 > 32) return fail(RF_EINVAL, "rf_diagnostics: too many variables");
    NODES_READY(c, "rf_diagnostics");
    DISPATCH(c, diagnostics(c, U, T, out, (cudaStream_t)s));
}

extern "C" int rf_set_option(rf_ctx *c, const char *key, double value) {
    if (!c || !key) return fail(RF_EINVAL, "rf_set_option: null argument");
    const int v = (int)value;
    if (!std::strcmp(key, "newton_maxit")) {
        if (v < 0 || v > 1000) return fail(RF_EINVAL, "rf_set_option: newton_maxit %d outside [0, 1000]", v);
        c->newton_maxit = v;
    } else if (!std::strcmp(key, "x_block")) {
        if (v < 32 || v > 256 || v % 32) return fail(RF_EINVAL, "rf_set_option: x_block %d not a multiple of 32 in [32, 256]", v);
        c->x_block = v;
    } else if (!std::strcmp(key, "walk_block")) {
        if (v < 32 || v > 128 || v % 32) return fail(RF_EINVAL, "rf_set_option: walk_block %d not a multiple of 32 in [32, 128]", v);
        c->walk_block = v;
    } else if (!std::strcmp(key, "profile")) {
        clear_profile(c);
        c->profile = v ? 1 : 0;
    } else if (!std::strcmp(key, "walk_seg")) {
        if (v < 1 || v > 4096) return fail(RF_EINVAL, "rf_set_option: walk_seg %d outside [1, 4096]", v);
        c->walk_seg = v;
        c->walk_seg_staged = v;
    } else {
        return fail(RF_EINVAL, "rf_set_option: unknown key '%s'", key);
    }
    return RF_OK;
}

template <typename R>
static int set_nodes_impl(rf_ctx *c, const double *nodes, cudaStream_t s) {
    const Nodes N{nodes, c->g.nx, c->g.ny, c->g.nz, (long long)(c->g.nx + 1) * (c->g.ny + 1) * (c->g.nz + 1)};
    unsigned long long *bad = (unsigned long long *)(c->gC + 3 * c->n);
    CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    const long long nf0 = (long long)geo_faces(c->g, 0), nf1 = (long long)geo_faces(c->g, 1), nf2 = (long long)geo_faces(c->g, 2);
    geometry_face_kernel<R, 0><<<(unsigned)((nf0 + 127) / 128), 128, 0, s>>>(N, (R *)c->gS[0]);
    geometry_face_kernel<R, 1><<<(unsigned)((nf1 + 127) / 128), 128, 0, s>>>(N, (R *)c->gS[1]);
    geometry_face_kernel<R, 2><<<(unsigned)((nf2 + 127) / 128), 128, 0, s>>>(N, (R *)c->gS[2]);
    geometry_cell_kernel<R><<<(unsigned)((c->n + 127) / 128), 128, 0, s>>>(N, (R *)c->gM, c->gV, (R *)c->giV, c->gC, bad);
    LAUNCH_CHECK();
    unsigned long long nbad = 0;
    CUDA_TRY(cudaMemcpyAsync(&nbad, bad, sizeof nbad, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (nbad) return fail(RF_EINVAL, "rf_set_nodes: %llu cells with a non-positive volume or a left-handed metric", nbad);
    c->nodes_set = 1;
    return RF_OK;
}

extern "C" int rf_set_nodes(rf_ctx *c, const double *nodes, rf_stream s) {
    if (!c || !nodes) return fail(RF_EINVAL, "rf_set_nodes: null argument");
    if (!(c->flags & RF_MAPPED)) return fail(RF_EINVAL, "rf_set_nodes: the context was not created with RF_MAPPED");
    c->nodes_set = 0;
    return c->precision == RF_FP64 ? set_nodes_impl<double>(c, nodes, (cudaStream_t)s)
                                   : set_nodes_impl<float>(c, nodes, (cudaStream_t)s);
}

extern "C" int rf_set_nscbc(rf_ctx *c, int axis, int side, const rf_nscbc *b) {
    if (!c || !b) return fail(RF_EINVAL, "rf_set_nscbc: null argument");
    if (axis < 0 || axis > 2) return fail(RF_EINVAL, "rf_set_nscbc: axis %d outside 0..2", axis);
    if (side != 0 && side != 1) return fail(RF_EINVAL, "rf_set_nscbc: side %d is neither 0 (low) nor 1 (high)", side);
    if (c->g.bc[axis] != RF_BC_NSCBC) return fail(RF_EINVAL, "rf_set_nscbc: axis %d is not an NSCBC axis (bc = %d)", axis, c->g.bc[axis]);
    const double co[6] = {b->p_inf, b->sigma, b->eta_u, b->eta_T, b->eta_t, b->eta_Y};
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(co[k])) return fail(RF_EINVAL, "rf_set_nscbc: non-finite coefficient");
    if (b->sigma < 0 || b->eta_u < 0 || b->eta_T < 0 || b->eta_t < 0 || b->eta_Y < 0)
        return fail(RF_EINVAL, "rf_set_nscbc: relaxation coefficients must be >= 0");
    if (!b->target && !(b->p_inf > 0)) return fail(RF_EINVAL, "rf_set_nscbc: an outflow side needs p_inf > 0");
    if (!std::isfinite(b->length)) return fail(RF_EINVAL, "rf_set_nscbc: non-finite length");
    c->nscbc[axis].s[side] = NscbcSide{b->p_inf, b->sigma, b->eta_u, b->eta_T, b->eta_t, b->eta_Y,
                                       b->length > 0 ? b->length : 0.0, b->target};
    ++c->nscbc_version;
    return RF_OK;
}

extern "C" int rf_profile_read(rf_ctx *c, double *ms, int *launches, int nclass) {
    if (!c || !ms || !launches || nclass < RF_NPROF) return fail(RF_EINVAL, "rf_profile_read: bad argument");
    for (int k = 0; k < RF_NPROF; ++k) {
        ms[k] = 0.0;
        launches[k] = (int)c->ev[k][1].size();
        for (size_t i = 0; i < c->ev[k][1].size(); ++i) {
            CUDA_TRY(cudaEventSynchronize(c->ev[k][1][i]));
            float e = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&e, c->ev[k][0][i], c->ev[k][1][i]));
            ms[k] += e;
        }
    }
    clear_profile(c);
    return RF_OK;
}

extern "C" int rf_status(rf_ctx *c, rf_stream s, long long *cell_out) {
    if (!c) return fail(RF_EINVAL, "rf_status: null context");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)s));
    int st = 0;
    long long cell = -1;
    CUDA_TRY(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&cell, c->bad_cell, sizeof(long long), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(c->status, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(c->bad_cell, 0xff, sizeof(long long)));
    if (cell_out) *cell_out = cell;
    if (st & ST_NONFINITE) return fail(RF_ENONFINITE, "non-finite state at cell %lld", cell);
    if (st & ST_NEWTON) return fail(RF_ENEWTON, "temperature Newton solve did not converge at cell %lld", cell);
    if (st & ST_RANGE) return fail(RF_ERANGE, "temperature or density out of range at cell %lld", cell);
    if (st & ST_TIMEOUT) return fail(RF_ETIMEOUT, "a bounded device wait gave up");
    return RF_OK;
}


// ----------------------------------------------------------------------------- ensembles

struct rf_ensemble {
    const rf_mech *mech = nullptr;
    int n = 0, precision = 0, ns = 0;
    bool all3d = true;
    bool any_mapped = false;                  // a mapped member: only the member loop (mode 0)
    std::vector<rf_ctx *> ctx;
    std::vector<double *> U, T;
    std::vector<rf_laser> las;
    double *t_dev = nullptr;
    Member *d_tab[3] = {nullptr, nullptr, nullptr};
    std::vector<Member> h_tab[3];             // host copies (launches of members' own kernels)
    long long nscbc_stamp = -1;               // members' NSCBC settings when the graphs were captured
    EnsItem *d_items[4] = {nullptr, nullptr, nullptr, nullptr};
    int nitems[4] = {0, 0, 0, 0};
    unsigned int *d_bar = nullptr;
    int *d_timeout = nullptr;
    int seg = 16, xblock = 128;
    long long max_spins = 20000000;          // ~2 s of polling per barrier
    unsigned int bar_extra = 0;              // tests: arrivals a barrier waits for beyond the grid
    size_t smem_cell = 0, smem_x = 0;
    int coop_blocks = 0;
    int mslot = 0;
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t graph_nodes[4] = {0, 0, 0, 0};
    cudaStream_t cap = nullptr;               // private stream for graph capture and replay
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;   // order the private stream after / before the caller's
};

static void ens_free_device(rf_ensemble *e) {
    for (int k = 0; k < 3; ++k)
        if (e->d_tab[k]) cudaFree(e->d_tab[k]), e->d_tab[k] = nullptr;
    for (int k = 0; k < 4; ++k)
        if (e->d_items[k]) cudaFree(e->d_items[k]), e->d_items[k] = nullptr;
    for (int k = 0; k < 4; ++k)
        if (e->graph[k]) cudaGraphExecDestroy(e->graph[k]), e->graph[k] = nullptr;
}

extern "C" void rf_ensemble_free(rf_ensemble *e) {
    if (!e) return;
    ens_free_device(e);
    if (e->d_bar) cudaFree(e->d_bar);
    if (e->d_timeout) cudaFree(e->d_timeout);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->ev_in) cudaEventDestroy(e->ev_in);
    if (e->ev_out) cudaEventDestroy(e->ev_out);
    delete e;
}

// x sweep row chunking for a block of B threads (see Path::sweep)
static void x_shape(int nx, int B, int &W, int &rpb) {
    if (nx <= B) {
        W = nx;
        rpb = std::max(1, std::min(B / nx, 320 / (nx + 2)));
    } else {
        W = B;
        rpb = 1;
    }
}

// (Re)builds the descriptor tables and work lists for the current seg / xblock.
static int ens_build(rf_ensemble *e) {
    ens_free_device(e);
    const double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0}, cc[3] = {0.0, 1.0, 0.5};
    std::vector<Member> tab[3];
    std::vector<EnsItem> items[4];
    size_t smx = 0;
    for (int mi = 0; mi < e->n; ++mi) {
        rf_ctx *c = e->ctx[mi];
        Member m = base_member(c);
        m.T = e->T[mi];
        m.Un = e->U[mi];
        set_laser(m, &e->las[mi]);
        int W, rpb;
        x_shape(c->g.nx, e->xblock, W, rpb);
        m.xW = W;
        m.xrpb = rpb;
        const double *in[3] = {e->U[mi], c->U1, c->U2};
        double *outp[3] = {c->U1, c->U2, e->U[mi]};
        for (int k = 0; k < 3; ++k) {
            Member mk = m;
            mk.U = in[k];
            mk.Uout = outp[k];
            mk.stage_a = a[k];
            mk.stage_b = b[k];
            mk.stage_c = cc[k];
            mk.want_rates = k == 0 ? 1 : 0;
            tab[k].push_back(mk);
        }
        const int nv = c->nv;
        const bool staged = c->precision == RF_MIXED;
        // staged x sweep (FP32 bulk): four rows per block, window buffers as XTile
        const size_t x_staged = x_staged_smem(c->ns);
        smx = std::max(smx, staged ? x_staged : (size_t)nv * rpb * (W + 2) * c->rsize);
        const long long ncb = (c->n + 127) / 128;
        for (long long q = 0; q < ncb; ++q) items[0].push_back({mi, (int)q, 0, 0});
        const int nrows = c->g.ny * c->g.nz;
        const int rows_per_item = staged ? 4 : rpb;
        for (int q = 0; q < (nrows + rows_per_item - 1) / rows_per_item; ++q) items[1].push_back({mi, q, 0, 0});
        for (int dir = 1; dir <= 2; ++dir) {
            const long long lines = (long long)c->g.nx * (dir == 1 ? c->g.nz : c->g.ny);
            const int nd = dir == 1 ? c->g.ny : c->g.nz;
            const int lb = (int)(c->precision == RF_MIXED ? walk_tiles<float, 1>(c->g.nx, dir == 1 ? c->g.nz : c->g.ny)
                                                          : walk_tiles<double, 1>(c->g.nx, dir == 1 ? c->g.nz : c->g.ny));
            const int sb = (nd + e->seg - 1) / e->seg;
            (void)lines;
            for (int q = 0; q < lb; ++q)
                for (int r = 0; r < sb; ++r) items[1 + dir].push_back({mi, q, r, 0});
        }
    }
    for (int k = 0; k < 3; ++k) {
        CUDA_TRY(cudaMalloc((void **)&e->d_tab[k], sizeof(Member) * e->n));
        CUDA_TRY(cudaMemcpy(e->d_tab[k], tab[k].data(), sizeof(Member) * e->n, cudaMemcpyHostToDevice));
        e->h_tab[k] = tab[k];
    }
    for (int k = 0; k < 4; ++k) {
        e->nitems[k] = (int)items[k].size();
        CUDA_TRY(cudaMalloc((void **)&e->d_items[k], sizeof(EnsItem) * std::max<size_t>(1, items[k].size())));
        CUDA_TRY(cudaMemcpy(e->d_items[k], items[k].data(), sizeof(EnsItem) * items[k].size(), cudaMemcpyHostToDevice));
    }
    e->smem_x = smx;
    return RF_OK;
}

static EnsDev ens_dev(rf_ensemble *e, unsigned int grid) {
    EnsDev E;
    std::memset(&E, 0, sizeof E);
    for (int k = 0; k < 3; ++k) E.tab[k] = e->d_tab[k];
    for (int k = 0; k < 4; ++k) {
        E.items[k] = e->d_items[k];
        E.nitems[k] = e->nitems[k];
    }
    E.nmembers = e->n;
    E.seg = e->seg;
    E.newton_maxit = e->ctx[0]->newton_maxit;
    E.bar = e->d_bar;
    E.timeout = e->d_timeout;
    E.max_spins = e->max_spins;
    E.bar_expect = grid + e->bar_extra;
    return E;
}

template <typename R, int NS>
struct EnsPath {
    using UT = typename std::conditional<sizeof(R) == 4, float, double>::type;

    // characteristic boundaries of the members that have NSCBC axes, each by its own
    // launches (a few planes of cells), after the stage's cell state
    static int members_nscbc(rf_ensemble *e, int k, cudaStream_t s) {
        for (int mi = 0; mi < e->n; ++mi) {
            rf_ctx *c = e->ctx[mi];
            if (c->g.bc[0] != RF_BC_NSCBC && c->g.bc[1] != RF_BC_NSCBC && c->g.bc[2] != RF_BC_NSCBC) continue;
            if (int rc = Path<R, NS>::nscbc(c, e->h_tab[k][mi], s)) return rc;
        }
        return RF_OK;
    }

    static int setup(rf_ensemble *e) {
        e->smem_cell = cell_state_smem_max<R, NS>(128, e->mech->nr);
        CUDA_TRY(cudaFuncSetAttribute(ens_cell_kernel<R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem_cell));
        CUDA_TRY(cudaFuncSetAttribute(ens_x_kernel<R, UT, NS, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)std::max<size_t>(e->smem_x, 1)));
        if constexpr (sizeof(R) == 4) {
            const int sw = (int)walk_smem<R, NS>();
            CUDA_TRY(cudaFuncSetAttribute(ens_walk_kernel<R, UT, NS, 1, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sw));
            CUDA_TRY(cudaFuncSetAttribute(ens_walk_kernel<R, UT, NS, 2, MODE_ACCUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sw));
        }
        const size_t sm_sweep = walk_smem<R, NS>();
        CUDA_TRY(cudaFuncSetAttribute(ens_sweep_stage_kernel<R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sweep));
        int dev = 0, sms = 0, per = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ens_sweep_stage_kernel<R, NS>, 128, sm_sweep));
        if (per < 1) return fail(RF_ECUDA, "ensemble: persistent sweep kernel does not fit on an SM");
        e->coop_blocks = per * sms;
        return RF_OK;
    }

    // one step as one launch per phase (mode 1/2)
    static int step_batched(rf_ensemble *e, cudaStream_t s) {
        const int M = e->mslot;
        for (int k = 0; k < 3; ++k) {
            EnsDev E0 = ens_dev(e, e->nitems[0]);
            ens_cell_kernel<R, NS><<<e->nitems[0], 128, cell_state_smem<R, NS>(128, k == 0, e->mech->nr), s>>>(M, E0, k);
            LAUNCH_CHECK();
            if (k == 0) {
                ens_dt_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(M, E0);
                LAUNCH_CHECK();
            }
            if (int rc = members_nscbc(e, k, s)) return rc;
            ens_x_kernel<R, UT, NS, MODE_ACCUM><<<e->nitems[1], 128, e->smem_x, s>>>(M, ens_dev(e, e->nitems[1]), k);
            LAUNCH_CHECK();
            ens_walk_kernel<R, UT, NS, 1, MODE_ACCUM><<<e->nitems[2], 128, walk_smem<R, NS>(), s>>>(M, ens_dev(e, e->nitems[2]), k);
            LAUNCH_CHECK();
            if constexpr (sizeof(R) == 4) {
                // FP32 bulk: the z sweep accumulates, an elementwise FP64 kernel applies the stage
                ens_walk_kernel<R, UT, NS, 2, MODE_ACCUM><<<e->nitems[3], 128, walk_smem<R, NS>(), s>>>(M, ens_dev(e, e->nitems[3]), k);
                LAUNCH_CHECK();
                ens_final_kernel<R, NS><<<e->nitems[0], 128, 0, s>>>(ens_dev(e, e->nitems[0]), k);
            } else {
                ens_walk_kernel<R, UT, NS, 2, MODE_STAGE><<<e->nitems[3], 128, walk_smem<R, NS>(), s>>>(M, ens_dev(e, e->nitems[3]), k);
            }
            LAUNCH_CHECK();
        }
        ens_end_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(ens_dev(e, 1));
        LAUNCH_CHECK();
        return RF_OK;
    }

    // one step as, per RK stage, work-list launches of the cell state (and, in the first
    // stage, the time step) and the x sweep, one cooperative launch of the y and z sweeps,
    // and (FP32 bulk) the stage update (mode 3)
    static int step_persistent(rf_ensemble *e, cudaStream_t s) {
        const size_t sm_sweep = walk_smem<R, NS>();
        const int M = e->mslot;
        for (int k = 0; k < 3; ++k) {
            EnsDev E0 = ens_dev(e, e->nitems[0]);
            ens_cell_kernel<R, NS><<<e->nitems[0], 128, cell_state_smem<R, NS>(128, k == 0, e->mech->nr), s>>>(M, E0, k);
            LAUNCH_CHECK();
            if (k == 0) {
                ens_dt_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(M, E0);
                LAUNCH_CHECK();
            }
            if (int rc = members_nscbc(e, k, s)) return rc;
            ens_x_kernel<R, UT, NS, MODE_ACCUM><<<e->nitems[1], 128, e->smem_x, s>>>(M, ens_dev(e, e->nitems[1]), k);
            LAUNCH_CHECK();
            EnsDev E = ens_dev(e, e->coop_blocks);
            cudaLaunchConfig_t cfg;
            std::memset(&cfg, 0, sizeof cfg);
            cfg.gridDim = dim3(e->coop_blocks);
            cfg.blockDim = dim3(128);
            cfg.dynamicSmemBytes = sm_sweep;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CUDA_TRY(cudaLaunchKernelEx(&cfg, ens_sweep_stage_kernel<R, NS>, e->mslot, E, k));
            if constexpr (sizeof(R) == 4) {
                ens_final_kernel<R, NS><<<e->nitems[0], 128, 0, s>>>(ens_dev(e, e->nitems[0]), k);
                LAUNCH_CHECK();
            }
        }
        ens_end_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(ens_dev(e, 1));
        LAUNCH_CHECK();
        return RF_OK;
    }
};

#define ENS_DISPATCH(e, CALL)                                                        \
    do {                                                                             \
        if ((e)->precision == RF_FP64) {                                             \
            switch ((e)->ns) {                                                       \
                case 1: return EnsPath<double, 1>::CALL;                             \
                case 2: return EnsPath<double, 2>::CALL;                             \
                case 4: return EnsPath<double, 4>::CALL;                             \
                case 9: return EnsPath<double, 9>::CALL;                             \
            }                                                                        \
        } else {                                                                     \
            switch ((e)->ns) {                                                       \
                case 1: return EnsPath<float, 1>::CALL;                              \
                case 2: return EnsPath<float, 2>::CALL;                              \
                case 4: return EnsPath<float, 4>::CALL;                              \
                case 9: return EnsPath<float, 9>::CALL;                              \
            }                                                                        \
        }                                                                            \
        return fail(RF_EINVAL, "unsupported species count %d", (e)->ns);             \
    } while (0)

static int ens_setup(rf_ensemble *e) { ENS_DISPATCH(e, setup(e)); }
static int ens_step_batched(rf_ensemble *e, cudaStream_t s) { ENS_DISPATCH(e, step_batched(e, s)); }
static int ens_step_persistent(rf_ensemble *e, cudaStream_t s) { ENS_DISPATCH(e, step_persistent(e, s)); }

extern "C" int rf_ensemble_create(rf_ctx *const *members, int n, double *const *U, double *const *T, const rf_laser *lasers,
                                  double *t_dev, rf_ensemble **out) {
    if (!members || !U || !T || !t_dev || !out || n < 1) return fail(RF_EINVAL, "rf_ensemble_create: bad argument");
    *out = nullptr;
    rf_ensemble *e = new rf_ensemble();
    e->n = n;
    e->t_dev = t_dev;
    for (int i = 0; i < n; ++i) {
        rf_ctx *c = members[i];
        if (!c || !U[i] || !T[i]) {
            delete e;
            return fail(RF_EINVAL, "rf_ensemble_create: member %d has a null context or buffer", i);
        }
        if ((c->flags & RF_MAPPED) && !c->nodes_set) {
            delete e;
            return fail(RF_EINVAL, "rf_ensemble_create: member %d is a mapped grid without node coordinates (rf_set_nodes)", i);
        }
        if (c->flags & RF_TENO6) {
            delete e;
            return fail(RF_EINVAL, "rf_ensemble_create: member %d uses TENO6; batched ensembles run WENO3-Z", i);
        }
        if (c->flags & RF_CHARWISE) {
            delete e;
            return fail(RF_EINVAL, "rf_ensemble_create: member %d uses RF_CHARWISE; batched ensembles run the component-wise splitting", i);
        }
        if (i == 0) {
            e->mech = c->mech;
            e->mslot = c->mslot;
            e->precision = c->precision;
            e->ns = c->ns;
        } else if (c->mech != e->mech || c->precision != e->precision) {
            delete e;
            return fail(RF_EINVAL, "rf_ensemble_create: member %d differs in mechanism or precision", i);
        }
        e->all3d = e->all3d && c->g.nx > 1 && c->g.ny > 1 && c->g.nz > 1;
        e->any_mapped = e->any_mapped || (c->flags & RF_MAPPED);
        e->ctx.push_back(c);
        e->U.push_back(U[i]);
        e->T.push_back(T[i]);
        rf_laser L;
        std::memset(&L, 0, sizeof L);
        if (lasers) L = lasers[i];
        e->las.push_back(L);
    }
    cudaError_t er = cudaMalloc((void **)&e->d_bar, 4 * sizeof(unsigned int));
    if (er == cudaSuccess) er = cudaMalloc((void **)&e->d_timeout, sizeof(int));
    if (er == cudaSuccess) er = cudaMemset(e->d_bar, 0, 4 * sizeof(unsigned int));
    if (er == cudaSuccess) er = cudaMemset(e->d_timeout, 0, sizeof(int));
    if (er == cudaSuccess) er = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
    if (er == cudaSuccess) er = cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming);
    if (er == cudaSuccess) er = cudaEventCreateWithFlags(&e->ev_out, cudaEventDisableTiming);
    if (er != cudaSuccess) {
        rf_ensemble_free(e);
        return fail(RF_ENOMEM, "rf_ensemble_create: %s", cudaGetErrorString(er));
    }
    int rc = ens_build(e);
    if (!rc) rc = ens_setup(e);
    if (rc) {
        rf_ensemble_free(e);
        return rc;
    }
    *out = e;
    return RF_OK;
}

extern "C" int rf_ensemble_set_option(rf_ensemble *e, const char *key, double value) {
    if (!e || !key) return fail(RF_EINVAL, "rf_ensemble_set_option: null argument");
    if (!std::strcmp(key, "walk_seg")) {
        if (value < 1 || value > 4096) return fail(RF_EINVAL, "rf_ensemble_set_option: walk_seg out of range");
        e->seg = (int)value;
        int rc = ens_build(e);
        return rc ? rc : ens_setup(e);
    }
    if (!std::strcmp(key, "barrier_spins")) {
        if (value < 1 || value > 1e9) return fail(RF_EINVAL, "rf_ensemble_set_option: barrier_spins out of range");
        e->max_spins = (long long)value;
    } else if (!std::strcmp(key, "barrier_extra")) {
        if (value < 0 || value > 1) return fail(RF_EINVAL, "rf_ensemble_set_option: barrier_extra must be 0 or 1");
        e->bar_extra = (unsigned int)value;
    } else {
        return fail(RF_EINVAL, "rf_ensemble_set_option: unknown key '%s'", key);
    }
    for (int k = 0; k < 4; ++k)
        if (e->graph[k]) cudaGraphExecDestroy(e->graph[k]), e->graph[k] = nullptr;
    return RF_OK;
}

static int ctx_rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl, const rf_laser *L,
                       cudaStream_t s) {
    DISPATCH(c, rk_step(c, U, T, t_dev, dt_fixed, cfl, L, nullptr, s));
}

static int ens_step(rf_ensemble *e, int mode, double cfl, double dt_fixed, cudaStream_t s) {
    if (mode == 0) {
        for (int i = 0; i < e->n; ++i) {
            int rc = ctx_rk_step(e->ctx[i], e->U[i], e->T[i], e->t_dev + i, dt_fixed, cfl, &e->las[i], s);
            if (rc) return rc;
        }
        return RF_OK;
    }
    if (mode >= 3) return ens_step_persistent(e, s);
    return ens_step_batched(e, s);
}

static int status_code(int st) {
    if (st & ST_TIMEOUT) return RF_ETIMEOUT;
    if (st & ST_NONFINITE) return RF_ENONFINITE;
    if (st & ST_NEWTON) return RF_ENEWTON;
    if (st & ST_RANGE) return RF_ERANGE;
    return RF_OK;
}

extern "C" int rf_run_ensemble(rf_ensemble *e, int nsteps, int mode, double cfl, double dt_fixed, int32_t *member_status,
                               rf_stream stream) {
    if (!e || nsteps < 0 || mode < 0 || mode > 3) return fail(RF_EINVAL, "rf_run_ensemble: bad argument");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(RF_EINVAL, "rf_run_ensemble: need dt_fixed > 0 or cfl > 0");
    if (mode > 0 && !e->all3d) return fail(RF_EINVAL, "rf_run_ensemble: batched modes need every member with nx, ny, nz > 1");
    if (mode > 0 && e->any_mapped)
        return fail(RF_EINVAL, "rf_run_ensemble: batched modes run Cartesian members; an ensemble with mapped members runs mode 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == 0) {
        for (int k = 0; k < nsteps; ++k) {
            int rc = ens_step(e, 0, cfl, dt_fixed, s);
            if (rc) return rc;
        }
    } else {
        CUDA_TRY(cudaMemsetAsync(e->d_timeout, 0, sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(e->d_bar, 0, 4 * sizeof(unsigned int), s));
        EnsDev E = ens_dev(e, 1);
        ens_begin_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(E, e->t_dev, cfl, dt_fixed);
        LAUNCH_CHECK();
        // modes 2 and 3 replay one step captured as a CUDA graph (mode 3's graph holds its
        // cooperative launches)
        const bool graph = mode == 2 || mode == 3;
        long long stamp = 0;
        for (rf_ctx *c : e->ctx) stamp += c->nscbc_version;
        if (stamp != e->nscbc_stamp) {
            // a member's boundary settings (captured as launch parameters) changed
            for (int q = 0; q < 4; ++q)
                if (e->graph[q]) cudaGraphExecDestroy(e->graph[q]), e->graph[q] = nullptr;
            e->nscbc_stamp = stamp;
        }
        if (graph && nsteps > 0 && !e->graph[mode]) {
            // captured on the ensemble's own stream: capture records, it does not run anything
            cudaGraph_t g;
            CUDA_TRY(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
            int rc = ens_step(e, mode, cfl, dt_fixed, e->cap);
            cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
            if (rc) return rc;
            if (ce != cudaSuccess) return fail(RF_ECUDA, "rf_run_ensemble: graph capture: %s", cudaGetErrorString(ce));
            size_t nodes = 0;
            cudaGraphGetNodes(g, nullptr, &nodes);
            cudaGraphExec_t ex = nullptr;
            ce = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess)
                return fail(RF_ECUDA, "rf_run_ensemble: graph instantiate (%zu nodes): %s", nodes, cudaGetErrorString(ce));
            if (!ex) return fail(RF_ECUDA, "rf_run_ensemble: graph instantiate returned no executable (%zu nodes)", nodes);
            e->graph[mode] = ex;
            e->graph_nodes[mode] = nodes;
        }
        if (graph && nsteps > 0) {
            // replay on the ensemble's stream, ordered after and before the caller's stream
            CUDA_TRY(cudaEventRecord(e->ev_in, s));
            CUDA_TRY(cudaStreamWaitEvent(e->cap, e->ev_in, 0));
            for (int k = 0; k < nsteps; ++k) {
                cudaError_t le = cudaGraphLaunch(e->graph[mode], e->cap);
                if (le != cudaSuccess) {
                    (void)cudaGetLastError();
                    return fail(RF_ECUDA, "rf_run_ensemble: cudaGraphLaunch (mode %d, %zu nodes, step %d): %s", mode,
                                e->graph_nodes[mode], k, cudaGetErrorString(le));
                }
            }
            CUDA_TRY(cudaEventRecord(e->ev_out, e->cap));
            CUDA_TRY(cudaStreamWaitEvent(s, e->ev_out, 0));
        } else {
            for (int k = 0; k < nsteps; ++k) {
                int rc = ens_step(e, mode, cfl, dt_fixed, s);
                if (rc) return rc;
            }
        }
        ens_finish_kernel<<<(e->n + 127) / 128, 128, 0, s>>>(E, e->t_dev);
        LAUNCH_CHECK();
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    int timeout = 0;
    CUDA_TRY(cudaMemcpy(&timeout, e->d_timeout, sizeof(int), cudaMemcpyDeviceToHost));
    int first = RF_OK;
    for (int i = 0; i < e->n; ++i) {
        rf_ctx *c = e->ctx[i];
        int st = 0;
        CUDA_TRY(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemset(c->status, 0, sizeof(int)));
        CUDA_TRY(cudaMemset(c->bad_cell, 0xff, sizeof(long long)));
        const int code = status_code(st);
        if (member_status) member_status[i] = code;
        if (code && !first) first = code;
    }
    if (timeout) {
        CUDA_TRY(cudaMemset(e->d_timeout, 0, sizeof(int)));
        return fail(RF_ETIMEOUT, "rf_run_ensemble: a grid barrier of the persistent kernel gave up waiting");
    }
    if (first && !member_status) return fail(first, "rf_run_ensemble: a member failed (pass member_status to mask it)");
    return RF_OK;
}

extern "C" int rf_ensemble_autotune(rf_ensemble *e, int mode, double cfl, int *seg_out, rf_stream stream) {
    if (!e || mode < 1 || mode > 3) return fail(RF_EINVAL, "rf_ensemble_autotune: bad argument");
    if (!e->all3d) return fail(RF_EINVAL, "rf_ensemble_autotune: batched modes need 3-D members");
    if (e->any_mapped) return fail(RF_EINVAL, "rf_ensemble_autotune: batched modes run Cartesian members");
    cudaStream_t s = (cudaStream_t)stream;
    // keep the states: trial steps run on them and are rolled back
    size_t tot = 0;
    for (int i = 0; i < e->n; ++i) tot += (size_t)e->ctx[i]->n * (e->ctx[i]->nv + 1);
    double *bk = nullptr;
    CUDA_TRY(cudaMalloc((void **)&bk, (tot + e->n) * sizeof(double)));
    auto copy_states = [&](bool save) -> int {
        size_t off = 0;
        for (int i = 0; i < e->n; ++i) {
            const size_t nu = (size_t)e->ctx[i]->n * e->ctx[i]->nv, nt = (size_t)e->ctx[i]->n;
            CUDA_TRY(cudaMemcpyAsync(save ? bk + off : e->U[i], save ? e->U[i] : bk + off, nu * 8, cudaMemcpyDeviceToDevice, s));
            off += nu;
            CUDA_TRY(cudaMemcpyAsync(save ? bk + off : e->T[i], save ? e->T[i] : bk + off, nt * 8, cudaMemcpyDeviceToDevice, s));
            off += nt;
        }
        CUDA_TRY(cudaMemcpyAsync(save ? bk + off : e->t_dev, save ? e->t_dev : bk + off, e->n * 8, cudaMemcpyDeviceToDevice, s));
        return RF_OK;
    };
    int rc = copy_states(true);
    const int cands[3] = {8, 16, 32};
    int best = e->seg;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int32_t> st(e->n);
    for (int q = 0; q < 3 && !rc; ++q) {
        rc = rf_ensemble_set_option(e, "walk_seg", cands[q]);
        if (rc) break;
        rc = rf_run_ensemble(e, 1, mode, cfl, 0.0, st.data(), stream);     // warm-up (and graph capture)
        if (rc) break;
        cudaEventRecord(e0, s);
        rc = rf_run_ensemble(e, 2, mode, cfl, 0.0, st.data(), stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && ms < best_ms) {
            best_ms = ms;
            best = cands[q];
        }
        if (!rc) rc = copy_states(false);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = rf_ensemble_set_option(e, "walk_seg", best);
    cudaStreamSynchronize(s);
    cudaFree(bk);
    if (seg_out) *seg_out = best;
    return rc;
}


// ----------------------------------------------------------------------------- adjoint

struct AdjWs {
    double *Qbar, *zero, *R, *lamS, *Ub1, *Ub2, *Ln, *T0, *T1, *T2;
};

static int adj_ws(rf_ctx *c, AdjWs &w) {
    if (c->flags & RF_TENO6) return fail(RF_EINVAL, "the discrete adjoint is built for WENO3-Z, not TENO6");
    if (c->flags & RF_CHARWISE) return fail(RF_EINVAL, "the discrete adjoint is built for the component-wise splitting, not RF_CHARWISE");
    if (c->flags & RF_MAPPED) return fail(RF_EINVAL, "the discrete adjoint is built for Cartesian grids, not RF_MAPPED ones");
    for (int a = 0; a < 3; ++a)
        if (c->g.bc[a] == RF_BC_NSCBC) return fail(RF_EINVAL, "the discrete adjoint is built for periodic and zero-gradient axes, not NSCBC (axis %d)", a);
    if (c->mech->npress > 0) return fail(RF_EINVAL, "the discrete adjoint is built for elementary reactions (the mechanism has %d pressure-dependent ones)", c->mech->npress);
    const size_t n = (size_t)c->n, nv = c->nv, nq = c->nq;
    const size_t tot = nq * n + 6 * nv * n + 3 * n;
    if (!c->adj) {
        cudaError_t e = cudaMalloc((void **)&c->adj, tot * sizeof(double));
        if (e != cudaSuccess) return fail(RF_ENOMEM, "adjoint workspace (%zu bytes): %s", tot * 8, cudaGetErrorString(e));
        c->bytes += tot * sizeof(double);
        CUDA_TRY(cudaMemset(c->adj, 0, tot * sizeof(double)));
    }
    double *p = c->adj;
    w.Qbar = p;
    p += nq * n;
    w.zero = p;
    p += nv * n;
    w.R = p;
    p += nv * n;
    w.lamS = p;
    p += nv * n;
    w.Ub1 = p;
    p += nv * n;
    w.Ub2 = p;
    p += nv * n;
    w.Ln = p;
    p += nv * n;
    w.T0 = p;
    p += n;
    w.T1 = p;
    p += n;
    w.T2 = p;
    return RF_OK;
}

static int axpby(double *y, const double *x, double a, double b, long long n, cudaStream_t s) {
    axpby_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, a, b, n);
    LAUNCH_CHECK();
    return RF_OK;
}

template <int NS>
struct AdjPath {
    static int adjoint_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, const double *lam,
                           double wH, double *lamU, double *grads, cudaStream_t s) {
        AdjWs w;
        int rc = adj_ws(c, w);
        if (rc) return rc;
        Member m = base_member(c);
        m.U = U;
        m.T = T;
        m.t_from_host = 1;
        m.t_host = t;
        set_laser(m, L);
        rc = Path<double, NS>::cell_state(c, m, s);        // Q and converged T of this state
        if (rc) return rc;
        CUDA_TRY(cudaMemsetAsync(w.Qbar, 0, (size_t)c->nq * c->n * sizeof(double), s));
        const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
        if (lam) {
            for (int d = 0; d < 3; ++d) {
                if (n3[d] <= 1) continue;
                const long long nf = (long long)(c->g.bc[d] == RF_BC_PERIODIC ? n3[d] : n3[d] + 1) * (c->n / n3[d]);
                const unsigned blocks = (unsigned)((nf + 127) / 128);
                if (d == 0) adjoint_face_kernel<NS, 0><<<blocks, 128, 0, s>>>(m, lam, lamU, w.Qbar);
                if (d == 1) adjoint_face_kernel<NS, 1><<<blocks, 128, 0, s>>>(m, lam, lamU, w.Qbar);
                if (d == 2) adjoint_face_kernel<NS, 2><<<blocks, 128, 0, s>>>(m, lam, lamU, w.Qbar);
                LAUNCH_CHECK();
            }
        }
        adjoint_cell_kernel<NS><<<(unsigned)((c->n + 63) / 64), 64, 0, s>>>(c->mslot, m, w.Qbar, lam ? lam : w.zero, lamU,
                                                                           grads, wH);
        LAUNCH_CHECK();
        return RF_OK;
    }

    // U_{n+1} from U_n through rhs evaluations and stage combinations (the same
    // arithmetic the adjoint step differentiates); *J += dt sum_k b_k H(U^(k)).
    // With `stages` (device, (2 nv + 3) n doubles) the step also keeps U^(1), U^(2), the
    // converged temperatures of U^n and U^(1) and the Newton warm start of U^(2) for
    // adjoint_step_stored.
    static int step_objective(rf_ctx *c, double *U, double *T, double t, double dt, const rf_laser *L, double *J,
                              cudaStream_t s, double *stages = nullptr) {
        AdjWs w;
        int rc = adj_ws(c, w);
        if (rc) return rc;
        const long long N = c->n * c->nv;
        const size_t tb = (size_t)c->n * 8;
        const double b[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
        const double *in[3] = {U, c->U1, c->U2};
        const double ts[3] = {t, t + dt, t + 0.5 * dt};
        double H[3];
        for (int k = 0; k < 3; ++k) {
            H[k] = 0.0;
            if (J) {           // the heat release only when the objective is requested
                rf_diag dg;
                rc = Path<double, NS>::diagnostics(c, in[k], T, &dg, s);
                if (rc) return rc;
                H[k] = dg.heat_release;
            }
            rc = Path<double, NS>::rhs(c, in[k], T, ts[k], L, w.R, s);
            if (rc) return rc;
            if (k == 0) {   // U1 = Un + dt R
                CUDA_TRY(cudaMemcpyAsync(c->U1, U, N * 8, cudaMemcpyDeviceToDevice, s));
                if ((rc = axpby(c->U1, w.R, dt, 1.0, N, s))) return rc;
                if (stages) {
                    CUDA_TRY(cudaMemcpyAsync(stages, c->U1, N * 8, cudaMemcpyDeviceToDevice, s));
                    CUDA_TRY(cudaMemcpyAsync(stages + 2 * N, T, tb, cudaMemcpyDeviceToDevice, s));
                }
            } else if (k == 1) {   // U2 = 3/4 Un + 1/4 (U1 + dt R)
                CUDA_TRY(cudaMemcpyAsync(c->U2, c->U1, N * 8, cudaMemcpyDeviceToDevice, s));
                if ((rc = axpby(c->U2, w.R, dt, 1.0, N, s))) return rc;
                if ((rc = axpby(c->U2, U, 0.75, 0.25, N, s))) return rc;
                if (stages) {
                    CUDA_TRY(cudaMemcpyAsync(stages + N, c->U2, N * 8, cudaMemcpyDeviceToDevice, s));
                    CUDA_TRY(cudaMemcpyAsync(stages + 2 * N + c->n, T, tb, cudaMemcpyDeviceToDevice, s));
                    CUDA_TRY(cudaMemcpyAsync(stages + 2 * N + 2 * c->n, T, tb, cudaMemcpyDeviceToDevice, s));
                }
            } else {   // Un+1 = 1/3 Un + 2/3 (U2 + dt R)
                if ((rc = axpby(c->U2, w.R, dt, 1.0, N, s))) return rc;
                if ((rc = axpby(U, c->U2, 2.0 / 3.0, 1.0 / 3.0, N, s))) return rc;
            }
        }
        if (J) *J += dt * (b[0] * H[0] + b[1] * H[1] + b[2] * H[2]);
        return RF_OK;
    }

    // lam <- (dU_{n+1}/dU_n)^T lam + wH dt sum_k b_k dH(U^(k))/dU_n; grads accumulate.
    static int adjoint_step(rf_ctx *c, const double *Un, const double *Tn, double t, double dt, const rf_laser *L,
                            double wH, double *lam, double *grads, cudaStream_t s) {
        AdjWs w;
        int rc = adj_ws(c, w);
        if (rc) return rc;
        const long long N = c->n * c->nv;
        // forward recompute: U1, U2 and the converged temperatures
        CUDA_TRY(cudaMemcpyAsync(w.T0, Tn, c->n * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = Path<double, NS>::rhs(c, Un, w.T0, t, L, w.R, s))) return rc;
        CUDA_TRY(cudaMemcpyAsync(c->U1, Un, N * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = axpby(c->U1, w.R, dt, 1.0, N, s))) return rc;
        CUDA_TRY(cudaMemcpyAsync(w.T1, w.T0, c->n * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = Path<double, NS>::rhs(c, c->U1, w.T1, t + dt, L, w.R, s))) return rc;
        CUDA_TRY(cudaMemcpyAsync(c->U2, c->U1, N * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = axpby(c->U2, w.R, dt, 1.0, N, s))) return rc;
        if ((rc = axpby(c->U2, Un, 0.75, 0.25, N, s))) return rc;
        CUDA_TRY(cudaMemcpyAsync(w.T2, w.T1, c->n * 8, cudaMemcpyDeviceToDevice, s));
        return adjoint_reverse(c, Un, c->U1, c->U2, w.T0, w.T1, w.T2, t, dt, L, wH, lam, grads, s);
    }

    // adjoint_step from the stage inputs step_objective kept in `stages` (their
    // temperatures serve as Newton warm starts and are overwritten).
    static int adjoint_step_stored(rf_ctx *c, const double *Un, double *stages, double t, double dt, const rf_laser *L,
                                   double wH, double *lam, double *grads, cudaStream_t s) {
        const long long N = c->n * c->nv;
        double *T0 = stages + 2 * N;
        return adjoint_reverse(c, Un, stages, stages + N, T0, T0 + c->n, T0 + 2 * c->n, t, dt, L, wH, lam, grads, s);
    }

    // The reverse of one step given its stage inputs U1, U2 and temperatures T0 (of Un),
    // T1 (of U1) and T2 (warm start of U2), each overwritten by the converged one.
    static int adjoint_reverse(rf_ctx *c, const double *Un, const double *U1, const double *U2, double *T0, double *T1,
                               double *T2, double t, double dt, const rf_laser *L, double wH, double *lam, double *grads,
                               cudaStream_t s) {
        AdjWs w;
        int rc = adj_ws(c, w);
        if (rc) return rc;
        const long long N = c->n * c->nv;
        // reverse: stage 3 (U2, t + dt/2)
        CUDA_TRY(cudaMemsetAsync(w.Ub2, 0, N * 8, s));
        CUDA_TRY(cudaMemsetAsync(w.lamS, 0, N * 8, s));
        if ((rc = axpby(w.lamS, lam, 2.0 / 3.0 * dt, 0.0, N, s))) return rc;
        if ((rc = adjoint_rhs(c, U2, T2, t + 0.5 * dt, L, w.lamS, wH * dt * (2.0 / 3.0), w.Ub2, grads, s))) return rc;
        if ((rc = axpby(w.Ub2, lam, 2.0 / 3.0, 1.0, N, s))) return rc;
        // stage 2 (U1, t + dt)
        CUDA_TRY(cudaMemsetAsync(w.Ub1, 0, N * 8, s));
        if ((rc = axpby(w.lamS, w.Ub2, 0.25 * dt, 0.0, N, s))) return rc;
        if ((rc = adjoint_rhs(c, U1, T1, t + dt, L, w.lamS, wH * dt / 6.0, w.Ub1, grads, s))) return rc;
        if ((rc = axpby(w.Ub1, w.Ub2, 0.25, 1.0, N, s))) return rc;
        // stage 1 (Un, t): lam_n = 1/3 lam + 3/4 Ub2 + Ub1 + VJP(Un, dt Ub1)
        CUDA_TRY(cudaMemcpyAsync(w.Ln, w.Ub1, N * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = axpby(w.Ln, w.Ub2, 0.75, 1.0, N, s))) return rc;
        if ((rc = axpby(w.Ln, lam, 1.0 / 3.0, 1.0, N, s))) return rc;
        if ((rc = axpby(w.lamS, w.Ub1, dt, 0.0, N, s))) return rc;
        if ((rc = adjoint_rhs(c, Un, T0, t, L, w.lamS, wH * dt / 6.0, w.Ln, grads, s))) return rc;
        CUDA_TRY(cudaMemcpyAsync(lam, w.Ln, N * 8, cudaMemcpyDeviceToDevice, s));
        return RF_OK;
    }
};

#define ADJ_DISPATCH(c, CALL)                                                        \
    do {                                                                             \
        if ((c)->precision != RF_FP64) return fail(RF_EINVAL, "adjoint: FP64 contexts only"); \
        switch ((c)->ns) {                                                           \
            case 1: return AdjPath<1>::CALL;                                         \
            case 2: return AdjPath<2>::CALL;                                         \
            case 4: return AdjPath<4>::CALL;                                         \
            case 9: return AdjPath<9>::CALL;                                         \
        }                                                                            \
        return fail(RF_EINVAL, "unsupported species count %d", (c)->ns);             \
    } while (0)

extern "C" int rf_adjoint_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, const double *lam_dUdt,
                              double w_hrr, double *lam_U, double *grad_params, rf_stream s) {
    if (!c || !U || !T || !lam_U || !grad_params) return fail(RF_EINVAL, "rf_adjoint_rhs: null argument");
    ADJ_DISPATCH(c, adjoint_rhs(c, U, T, t, L, lam_dUdt, w_hrr, lam_U, grad_params, (cudaStream_t)s));
}

extern "C" int rf_rk_step_objective(rf_ctx *c, double *U, double *T, double t, double dt, const rf_laser *L, double *J,
                                    rf_stream s) {
    if (!c || !U || !T || !(dt > 0.0)) return fail(RF_EINVAL, "rf_rk_step_objective: bad argument");
    ADJ_DISPATCH(c, step_objective(c, U, T, t, dt, L, J, (cudaStream_t)s));
}

extern "C" int rf_adjoint_rk_step(rf_ctx *c, const double *Un, const double *Tn, double t, double dt, const rf_laser *L,
                                  double w_hrr, double *lam, double *grad_params, rf_stream s) {
    if (!c || !Un || !Tn || !lam || !grad_params || !(dt > 0.0)) return fail(RF_EINVAL, "rf_adjoint_rk_step: bad argument");
    ADJ_DISPATCH(c, adjoint_step(c, Un, Tn, t, dt, L, w_hrr, lam, grad_params, (cudaStream_t)s));
}

extern "C" int rf_rk_step_stages(rf_ctx *c, double *U, double *T, double t, double dt, const rf_laser *L, double *J,
                                 double *stages, rf_stream s) {
    if (!c || !U || !T || !stages || !(dt > 0.0)) return fail(RF_EINVAL, "rf_rk_step_stages: bad argument");
    ADJ_DISPATCH(c, step_objective(c, U, T, t, dt, L, J, (cudaStream_t)s, stages));
}

extern "C" int rf_adjoint_rk_step_stored(rf_ctx *c, const double *Un, double *stages, double t, double dt,
                                         const rf_laser *L, double w_hrr, double *lam, double *grad_params, rf_stream s) {
    if (!c || !Un || !stages || !lam || !grad_params || !(dt > 0.0))
        return fail(RF_EINVAL, "rf_adjoint_rk_step_stored: bad argument");
    ADJ_DISPATCH(c, adjoint_step_stored(c, Un, stages, t, dt, L, w_hrr, lam, grad_params, (cudaStream_t)s));
}

// ----------------------------------------------------------------------------- peak probe

// Eight independent FMA chains per thread on every SM: the issue-limited FMA rate
// of the type, the ALU roofline of the FP64-bound cell-state kernel.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T *out, int iters, T b, T c) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += a[k];
    if (sum == (T)-1.25) out[0] = sum;        // keeps the chains live; never true
}

extern "C" int rf_probe_peak(int kind, double *tflops, rf_stream s) {
    if (!tflops || (kind != 0 && kind != 1)) return fail(RF_EINVAL, "rf_probe_peak: bad argument");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    const int iters = kind == 0 ? 2048 : 65536;
    cudaStream_t st = (cudaStream_t)s;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {        // first launch warms up
        CUDA_TRY(cudaEventRecord(e0, st));
        if (kind == 0) fma_probe_kernel<double><<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999, 1e-9);
        else fma_probe_kernel<float><<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999f, 1e-9f);
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return RF_OK;
}

__global__ void exp_pair_probe_kernel(const double *x, double *ep, double *em, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) exp_pair(x[i], ep[i], em[i]);
}

__global__ void math_probe_kernel(int fn, const double *x, double *y, double *y2, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (fn == 0) exp_pair(x[i], y[i], y2[i]);
    else if (fn == 1) y[i] = log64(x[i]);
    else if (fn == 2) y[i] = exp64(x[i]);
    else if (fn == 5) exp_pair_mixed(x[i], y[i], y2[i]);
    else if (fn == 6) y[i] = log64_mixed(x[i]);
    else if (fn == 3) {
        y[i] = (double)d2f(x[i]);
        y2[i] = (double)(float)x[i];
    } else {
        const float f = __uint_as_float((unsigned)__double2loint(x[i]));
        y[i] = f2d(f);
        y2[i] = (double)f;
    }
}

extern "C" int rf_probe_math(int fn, const double *x, double *y, double *y2, long long n, rf_stream s) {
    if (fn < 0 || fn > 6 || n < 0 || (n > 0 && (!x || !y || ((fn == 0 || (fn >= 3 && fn <= 5)) && !y2))))
        return fail(RF_EINVAL, "rf_probe_math: bad argument");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= RF_MAX_DEVICES) return fail(RF_EINVAL, "device %d out of range", dev);
    {
        std::lock_guard<std::mutex> lock(g_slot_mutex);
        if (int rc = upload_exp_table(dev)) return rc;
    }
    if (n == 0) return RF_OK;
    math_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)s>>>(fn, x, y, y2, n);
    LAUNCH_CHECK();
    return RF_OK;
}

// ----------------------------------------------------------------------------- allocation-free RHS

// Scratch of rf_rhs_noalloc: a file-scope device array, so the entry point never
// allocates.  Each GPU that loads this library holds these bytes until the
// process exits.  In host code `g_noalloc_scratch` names a host-side stand-in,
// not the device array: its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
static constexpr size_t RF_NOALLOC_BYTES = (size_t)16 << 20;
static constexpr size_t RF_NOALLOC_HEADER = 256;   // status, bad cell, clock, rate maxima
static __device__ __align__(256) unsigned char g_noalloc_scratch[RF_NOALLOC_BYTES];
static constexpr int RF_NOALLOC_MAX_DEVICES = 64;
static unsigned char *g_noalloc_dev[RF_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int noalloc_rhs_dispatch(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, double *dUdt,
                                cudaStream_t s) {
    DISPATCH(c, rhs(c, U, T, t, L, dUdt, s));
}

extern "C" int rf_rhs_noalloc(const rf_mech *m, const rf_grid_desc *g, int precision, uint32_t flags, const double *U,
                              double *T, double t, const rf_laser *L, double *dUdt, rf_stream s) {
    if (!m || !g || !U || !T || !dUdt) return fail(RF_EINVAL, "rf_rhs_noalloc: null argument");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(RF_EINVAL, "rf_rhs_noalloc: grid %dx%dx%d has an empty axis", g->nx, g->ny, g->nz);
    if (g->nx > 1024) return fail(RF_EINVAL, "rf_rhs_noalloc: nx = %d exceeds 1024", g->nx);
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return fail(RF_EINVAL, "rf_rhs_noalloc: grid spacing must be > 0");
    for (int a = 0; a < 3; ++a) {
        if (g->bc[a] == RF_BC_NSCBC)
            return fail(RF_EINVAL, "rf_rhs_noalloc: bc[%d] is NSCBC, whose side settings live in a context (rf_set_nscbc)", a);
        if (g->bc[a] != RF_BC_PERIODIC && g->bc[a] != RF_BC_EXTRAPOLATE) return fail(RF_EINVAL, "rf_rhs_noalloc: bc[%d] = %d unknown", a, g->bc[a]);
    }
    if (precision != RF_FP64 && precision != RF_MIXED) return fail(RF_EINVAL, "rf_rhs_noalloc: precision %d unknown", precision);
    if (flags & ~(uint32_t)RF_FLAGS_ALL) return fail(RF_EINVAL, "rf_rhs_noalloc: unknown flag bits 0x%x", flags & ~(uint32_t)RF_FLAGS_ALL);
    if (flags & RF_MAPPED) return fail(RF_EINVAL, "rf_rhs_noalloc: RF_MAPPED needs a context (rf_set_nodes)");
    if (flags & RF_CHARWISE) return fail(RF_EINVAL, "rf_rhs_noalloc: RF_CHARWISE runs through a context");
    const long long n = (long long)g->nx * g->ny * g->nz;
    const int ns = m->ns, nv = ns + 4, nq = Q_X0 + 3 * ns;
    const size_t rsize = precision == RF_FP64 ? sizeof(double) : sizeof(float);
    const size_t bq = align256((size_t)n * nq * rsize), br = align256((size_t)n * nv * rsize);
    const size_t b32 = precision == RF_MIXED ? align256((size_t)n * nv * sizeof(float)) : 0;
    const size_t need = RF_NOALLOC_HEADER + bq + br + b32;
    if (need > RF_NOALLOC_BYTES)
        return fail(RF_EINVAL, "rf_rhs_noalloc: grid of %lld cells needs %zu scratch bytes, more than the %zu-byte maximum",
                    n, need, RF_NOALLOC_BYTES);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= RF_NOALLOC_MAX_DEVICES) return fail(RF_EINVAL, "rf_rhs_noalloc: device %d out of range", dev);
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_dev[dev]) {
            void *p = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_dev[dev] = (unsigned char *)p;
        }
        base = g_noalloc_dev[dev];
    }
    int mslot = 0;
    {
        int rc = mech_slot(m, &mslot);
        if (rc) return rc;
    }
    cudaStream_t st = (cudaStream_t)s;
    // the header persists between calls: clear the status word, reset the bad-cell index
    CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(int) * 2, st));
    CUDA_TRY(cudaMemsetAsync(base + 8, 0xff, sizeof(long long), st));
    rf_ctx c;                                  // descriptor only: every buffer points into the scratch
    c.mech = m;
    c.mslot = mslot;
    c.g = *g;
    c.precision = precision;
    c.flags = flags;
    c.n = n;
    c.ns = ns;
    c.nv = nv;
    c.nq = nq;
    c.rsize = rsize;
    c.status = (int *)base;
    c.bad_cell = (long long *)(base + 8);
    c.clock = (double *)(base + 64);
    c.rates = (unsigned long long *)(base + 128);
    c.Q = base + RF_NOALLOC_HEADER;
    c.rhs = base + RF_NOALLOC_HEADER + bq;
    c.U32 = precision == RF_MIXED ? (float *)(base + RF_NOALLOC_HEADER + bq + br) : nullptr;
    {
        // kernel attributes once per device, precision and species count
        static std::mutex mu;
        static bool done[RF_NOALLOC_MAX_DEVICES][2][NSMAX + 1];
        std::lock_guard<std::mutex> lock(mu);
        bool &d = done[dev][precision == RF_MIXED ? 1 : 0][ns];
        if (!d) {
            if (int rc = prepare_ctx(&c)) return rc;
            d = true;
        }
    }
    int rc = noalloc_rhs_dispatch(&c, U, T, t, L, dUdt, st);
    if (rc) return rc;
    int status = 0;
    long long cell = -1;
    CUDA_TRY(cudaMemcpyAsync(&status, base, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&cell, base + 8, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (status & ST_NONFINITE) return fail(RF_ENONFINITE, "non-finite state at cell %lld", cell);
    if (status & ST_NEWTON) return fail(RF_ENEWTON, "temperature Newton solve did not converge at cell %lld", cell);
    if (status & ST_RANGE) return fail(RF_ERANGE, "temperature or density out of range at cell %lld", cell);
    return RF_OK;
}
