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
#include "rf_kernels.cuh"

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
            return fail(e_ == cudaErrorMemoryAllocation ? RF_ENOMEM : RF_ECUDA, "%s: %s (%s:%d)", #call, \
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

struct rf_mech {
    MechDev d;
    int ns, nr;
};

enum { PROF_CELL = 0, PROF_SWEEP_X = 1, PROF_SWEEP_Y = 2, PROF_SWEEP_Z = 3, PROF_OTHER = 4, RF_NPROF = 5 };

struct rf_ctx {
    const rf_mech *mech;
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
    int walk_block = 128, walk_seg = 16;     // y / z sweeps
    size_t bytes = 0;
    // optional per-kernel timing: CUDA events recorded on the launching stream
    int profile = 0;
    std::vector<cudaEvent_t> ev[RF_NPROF][2];
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
            M.sc[r][s][0] = a[0];
            M.sc[r][s][1] = a[1];
            M.sc[r][s][2] = a[2] / 2.0;
            M.sc[r][s][3] = a[3] / 3.0;
            M.sc[r][s][4] = a[4] / 4.0;
            M.sc[r][s][5] = a[6];
            M.gc[r][s][0] = a[0] - a[6];
            M.gc[r][s][1] = -a[1] / 2.0;
            M.gc[r][s][2] = -a[2] / 6.0;
            M.gc[r][s][3] = -a[3] / 12.0;
            M.gc[r][s][4] = -a[4] / 20.0;
            M.gc[r][s][5] = a[5];
            M.gc[r][s][6] = -a[0];
            for (int k = 0; k < 5; ++k) M.cpcf[r][s][k] = (float)a[k];
            for (int k = 0; k < 6; ++k) M.ecf[r][s][k] = (float)M.ec[r][s][k];
        }
        M.mu_ref[s] = d->mu_ref[s];
        M.mu_exp[s] = d->mu_exp[s];
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
        M.n_prod[j] = (int8_t)npd;
        M.n_net[j] = (int8_t)nnet;
        M.dnu_sum[j] = (int8_t)dsum;
    }
    *out = m;
    return RF_OK;
}

extern "C" void rf_free_mechanism(rf_mech *m) { delete m; }

static void free_ctx_buffers(rf_ctx *c) {
    void *ptrs[] = {c->Q, c->rhs, c->U32, c->U1, c->U2, c->clock, c->rates, c->status, c->bad_cell, c->diag};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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

extern "C" int rf_create_ctx(const rf_mech *m, const rf_grid_desc *g, int precision, uint32_t flags, rf_ctx **out) {
    if (!m || !g || !out) return fail(RF_EINVAL, "rf_create_ctx: null argument");
    *out = nullptr;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(RF_EINVAL, "rf_create_ctx: grid %dx%dx%d has an empty axis", g->nx, g->ny, g->nz);
    if (g->nx > 1024) return fail(RF_EINVAL, "rf_create_ctx: nx = %d exceeds 1024", g->nx);
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return fail(RF_EINVAL, "rf_create_ctx: grid spacing must be > 0");
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] != RF_BC_PERIODIC && g->bc[a] != RF_BC_EXTRAPOLATE) return fail(RF_EINVAL, "rf_create_ctx: bc[%d] = %d unknown", a, g->bc[a]);
    if (precision != RF_FP64 && precision != RF_MIXED) return fail(RF_EINVAL, "rf_create_ctx: precision %d unknown", precision);
    rf_ctx *c = new rf_ctx();
    c->mech = m;
    c->g = *g;
    c->precision = precision;
    c->flags = flags;
    c->n = (long long)g->nx * g->ny * g->nz;
    c->ns = m->ns;
    c->nv = m->ns + 4;
    c->nq = Q_X0 + 3 * m->ns;
    c->rsize = precision == RF_FP64 ? sizeof(double) : sizeof(float);
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
    m.n = c->n;
    m.Q = c->Q;
    m.rhs = c->rhs;
    m.U32 = c->U32;
    m.clock = c->clock;
    m.rates = c->rates;
    m.status = c->status;
    m.bad_cell = c->bad_cell;
    m.flags = (int)c->flags;
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
    }
}

template <typename R, int NS>
struct Path {
    using UT = typename std::conditional<sizeof(R) == 4, float, double>::type;

    static int cell_state(rf_ctx *c, const Member &m, cudaStream_t s) {
        const int B = 128;
        const long long nb = (c->n + B - 1) / B;
        const size_t smem = (size_t)B * NS * (3 * sizeof(double) + 2 * sizeof(R) + (sizeof(R) == 4 ? sizeof(R) : 0));
        ProfScope ps(c, PROF_CELL, s);
        cell_state_kernel<R, NS><<<(unsigned)nb, B, smem, s>>>(c->mech->d, m, c->newton_maxit);
        LAUNCH_CHECK();
        return RF_OK;
    }

    template <int MODE>
    static int sweep(rf_ctx *c, const Member &m, int dir, cudaStream_t s) {
        constexpr int NV = NS + 4;
        if (dir == 0) {
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
            sweep_x_kernel<R, UT, NS, MODE><<<blocks, threads, smem, s>>>(c->mech->d, m, W, rpb);
        } else {
            const int nd = dir == 1 ? c->g.ny : c->g.nz;
            const long long lines = (long long)c->g.nx * (dir == 1 ? c->g.nz : c->g.ny);
            dim3 grid((unsigned)((lines + c->walk_block - 1) / c->walk_block), (unsigned)((nd + c->walk_seg - 1) / c->walk_seg));
            ProfScope ps(c, dir == 1 ? PROF_SWEEP_Y : PROF_SWEEP_Z, s);
            if (dir == 1)
                sweep_walk_kernel<R, UT, NS, 1, MODE><<<grid, c->walk_block, 0, s>>>(c->mech->d, m, c->walk_seg);
            else
                sweep_walk_kernel<R, UT, NS, 2, MODE><<<grid, c->walk_block, 0, s>>>(c->mech->d, m, c->walk_seg);
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
        for (int d = 0; d < 3; ++d) {
            if (n[d] <= 1) continue;
            int rc = d == last ? sweep<MODE>(c, m, d, s) : sweep<MODE_ACCUM>(c, m, d, s);
            if (rc) return rc;
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
        return sweeps<MODE_RHS>(c, m, s);
    }

    static int rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl, const rf_laser *L,
                       double *dt_dev, cudaStream_t s) {
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
        const double hmin = std::min(c->g.nx > 1 ? c->g.dx : 1e300,
                                     std::min(c->g.ny > 1 ? c->g.dy : 1e300, c->g.nz > 1 ? c->g.dz : 1e300));
        for (int k = 0; k < 3; ++k) {
            m.U = in[k];
            m.Uout = outp[k];
            m.stage_a = a[k];
            m.stage_b = b[k];
            m.stage_c = cc[k];
            m.want_rates = (k == 0 && !(dt_fixed > 0.0)) ? 1 : 0;
            int rc = cell_state(c, m, s);
            if (rc) return rc;
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
        init_state_kernel<NS><<<(unsigned)((c->n + 127) / 128), 128, 0, s>>>(c->mech->d, prim, U, T, c->n);
        LAUNCH_CHECK();
        return RF_OK;
    }

    static int diagnostics(rf_ctx *c, const double *U, double *T, rf_diag *out, cudaStream_t s) {
        Member m = base_member(c);
        m.U = U;
        m.T = T;
        const int B = 64;
        const size_t smem = (size_t)B * NS * 5 * sizeof(double);
        diag_kernel<NS><<<c->diag_blocks, B, smem, s>>>(c->mech->d, m, c->diag, c->newton_maxit);
        LAUNCH_CHECK();
        const int nvals = NS + 6;
        double *res = c->diag + (size_t)c->diag_blocks * nvals;
        diag_fold_kernel<<<1, 32, 0, s>>>(c->diag, c->diag_blocks, nvals, res);
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

extern "C" int rf_init_state(rf_ctx *c, const double *prim, double *U, double *T, rf_stream s) {
    if (!c || !prim || !U || !T) return fail(RF_EINVAL, "rf_init_state: null argument");
    DISPATCH(c, init_state(c, prim, U, T, (cudaStream_t)s));
}

extern "C" int rf_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *L, double *dUdt, rf_stream s) {
    if (!c || !U || !T || !dUdt) return fail(RF_EINVAL, "rf_rhs: null argument");
    DISPATCH(c, rhs(c, U, T, t, L, dUdt, (cudaStream_t)s));
}

extern "C" int rf_rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl, const rf_laser *L,
                          double *dt_dev, rf_stream s) {
    if (!c || !U || !T || !t_dev) return fail(RF_EINVAL, "rf_rk_step: null argument");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(RF_EINVAL, "rf_rk_step: need dt_fixed > 0 or cfl > 0");
    DISPATCH(c, rk_step(c, U, T, t_dev, dt_fixed, cfl, L, dt_dev, (cudaStream_t)s));
}

extern "C" int rf_diagnostics(rf_ctx *c, const double *U, double *T, rf_diag *out, rf_stream s) {
    if (!c || !U || !T || !out) return fail(RF_EINVAL, "rf_diagnostics: null argument");
    if (c->nv + 2 > 32) return fail(RF_EINVAL, "rf_diagnostics: too many variables");
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
    } else {
        return fail(RF_EINVAL, "rf_set_option: unknown key '%s'", key);
    }
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
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] != RF_BC_PERIODIC && g->bc[a] != RF_BC_EXTRAPOLATE) return fail(RF_EINVAL, "rf_rhs_noalloc: bc[%d] = %d unknown", a, g->bc[a]);
    if (precision != RF_FP64 && precision != RF_MIXED) return fail(RF_EINVAL, "rf_rhs_noalloc: precision %d unknown", precision);
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
    cudaStream_t st = (cudaStream_t)s;
    // the header persists between calls: clear the status word, reset the bad-cell index
    CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(int) * 2, st));
    CUDA_TRY(cudaMemsetAsync(base + 8, 0xff, sizeof(long long), st));
    rf_ctx c;                                  // descriptor only: every buffer points into the scratch
    c.mech = m;
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
