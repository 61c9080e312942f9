// Batched ensembles: many members (grids of uneven size, each with its own laser
// and workspace) advanced together.  Every phase of an RK stage (cell state, x,
// y, z sweeps, time step) becomes one launch over a work list of (member, tile)
// items spanning all members; the "persistent" form runs the y and z sweeps of a stage
// in one cooperative launch whose blocks stride over the work lists and meet at a grid
// barrier between the phases, the other phases as such launches.  Results of a
// member are bitwise those of running it alone: every cell sees the same arithmetic
// whatever block processes it.
#pragma once

#include "rf_kernels.cuh"

namespace rf {

struct EnsItem {
    int m;    // member
    int a;    // tile index (cell block, row group or line block)
    int b;    // segment index (y / z sweeps)
    int pad;
};

struct EnsDev {
    const Member *tab[3];        // member descriptors of stages 1, 2, 3
    const EnsItem *items[4];     // cell state, x, y, z work lists
    int nitems[4];
    int nmembers;
    int seg;                     // cells walked per thread in the y / z sweeps
    int newton_maxit;
    unsigned int *bar;           // [0] arrivals, [1] generation, [2] / [3] next y / z item of the
                                 // persistent sweep launch
    int *timeout;                // set when a grid barrier gives up
    long long max_spins;         // bound on a barrier wait (iterations of ~100 ns)
    unsigned int bar_expect;     // blocks a barrier waits for (gridDim.x; larger only in tests)
};

// One thread per member: dt from the member's rate maxima (time-step rule).
__device__ __forceinline__ void member_dt(const MechDev &M, const Member &m) {
    double *clock = m.clock;
    double dt = clock[3];
    if (!(dt > 0.0)) {
        const double ac = __longlong_as_double((long long)m.rates[0]);
        const double df = __longlong_as_double((long long)m.rates[1]);
        const double ch = __longlong_as_double((long long)m.rates[2]);
        double hmin = 1e300;
        if (m.nx > 1) hmin = fmin(hmin, m.h[0]);
        if (m.ny > 1) hmin = fmin(hmin, m.h[1]);
        if (m.nz > 1) hmin = fmin(hmin, m.h[2]);
        dt = ac > 0.0 ? clock[2] / ac : 1.0e300;
        if (!(m.flags & F_NO_VISCOUS) && df > 0.0) dt = fmin(dt, 0.25 * hmin * hmin / df);
        if (!(m.flags & F_NO_CHEM) && M.nr > 0 && ch > 0.0) dt = fmin(dt, 0.2 / ch);
        if (m.laser_on && !(m.flags & F_NO_LASER)) {
            const double t = clock[0];
            const double lo = m.las[5] - 6.0 * m.las[6], hi = m.las[5] + 6.0 * m.las[6];
            if (t + dt > lo && t < hi) dt = fmin(dt, fmax(0.25 * m.las[6], lo - t));
        }
    }
    clock[1] = dt;
}

// Loads member descriptor it.m into shared memory, eight bytes per thread; returns
// false (uniformly) if the member has failed and must be skipped.
static_assert(sizeof(Member) % 8 == 0 && sizeof(Member) / 8 <= 128, "Member copy layout");
__device__ __forceinline__ bool load_member(const Member *tab, int mi, Member &sm, int &s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) s_ok = (*(volatile int *)tab[mi].status) == 0;
    if (threadIdx.x < sizeof(Member) / 8)
        reinterpret_cast<long long *>(&sm)[threadIdx.x] = reinterpret_cast<const long long *>(tab + mi)[threadIdx.x];
    __syncthreads();
    return s_ok != 0;
}

template <typename R, int NS>
__device__ __forceinline__ void ens_cell_phase(const MechDev &M, const EnsDev &E, int stage, unsigned char *smem,
                                               Member &sm, int &s_ok) {
    for (int w = blockIdx.x; w < E.nitems[0]; w += gridDim.x) {
        const EnsItem it = E.items[0][w];
        if (!load_member(E.tab[stage], it.m, sm, s_ok)) continue;
        cell_state_block<R, NS>(M, sm, it.a, smem, E.newton_maxit);
    }
}

template <typename R, typename UT, int NS, int MODE>
__device__ __forceinline__ void ens_x_phase(const MechDev &M, const EnsDev &E, int stage, unsigned char *smem, Member &sm,
                                            int &s_ok) {
    for (int w = blockIdx.x; w < E.nitems[1]; w += gridDim.x) {
        const EnsItem it = E.items[1][w];
        if (!load_member(E.tab[stage], it.m, sm, s_ok)) continue;
        if constexpr (sizeof(R) == 4)
            sweep_x_staged_block<NS, MODE>(M, sm, it.a, (float *)smem);
        else
            sweep_x_block<R, UT, NS, MODE>(M, sm, it.a, sm.xW, sm.xrpb, smem);
    }
}

// Elementwise FP64 stage update over the cell-state work list (FP32-bulk path: every
// sweep accumulates, then U_out = a Un + b (U + dt L), as in a single-grid stage).
template <typename R, int NS>
__device__ __forceinline__ void ens_final_phase(const EnsDev &E, int stage, Member &sm, int &s_ok) {
    for (int w = blockIdx.x; w < E.nitems[0]; w += gridDim.x) {
        const EnsItem it = E.items[0][w];
        if (!load_member(E.tab[stage], it.m, sm, s_ok)) continue;
        const long long cell = sm.c_lo + (long long)it.a * blockDim.x + threadIdx.x;
        if (cell < sm.c_hi) {
            R z[NS + 4];
#pragma unroll
            for (int v = 0; v < NS + 4; ++v) z[v] = 0;
            cell_update<R, NS, MODE_STAGE>(sm, cell, z, R(0));
        }
    }
}

// y / z work items: (tile, segment); a tile is a 32 x 4 line group of the staged
// walk in the FP32-bulk path and a block of 128 lines otherwise.
template <typename R, typename UT, int NS, int DIR, int MODE>
__device__ __forceinline__ void ens_walk_phase(const MechDev &M, const EnsDev &E, int stage, unsigned char *smem,
                                               Member &sm, int &s_ok) {
    const int k = DIR == 1 ? 2 : 3;
    for (int w = blockIdx.x; w < E.nitems[k]; w += gridDim.x) {
        const EnsItem it = E.items[k][w];
        if (!load_member(E.tab[stage], it.m, sm, s_ok)) continue;
        if constexpr (sizeof(R) == 4)
            sweep_walk_staged_block<NS, DIR, MODE>(M, sm, it.a, it.b, E.seg, (float *)smem);
        else
            sweep_walk_block<R, UT, NS, DIR, MODE>(M, sm, it.a, it.b, E.seg);
    }
}

// The same phase with dynamic work assignment: each block takes the next item from the
// counter E.bar[k] (k = 2 for y, 3 for z) until the list is exhausted, so that blocks
// that drew short items (members' ragged edges) take more; the items and their
// arithmetic are those of ens_walk_phase.
template <typename R, typename UT, int NS, int DIR, int MODE>
__device__ __forceinline__ void ens_walk_phase_dynamic(const MechDev &M, const EnsDev &E, int stage, unsigned char *smem,
                                                       Member &sm, int &s_ok, int &s_w) {
    const int k = DIR == 1 ? 2 : 3;
    for (;;) {
        if (threadIdx.x == 0) s_w = (int)atomicAdd(E.bar + k, 1u);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= E.nitems[k]) break;
        const EnsItem it = E.items[k][w];
        if (!load_member(E.tab[stage], it.m, sm, s_ok)) continue;
        if constexpr (sizeof(R) == 4)
            sweep_walk_staged_block<NS, DIR, MODE>(M, sm, it.a, it.b, E.seg, (float *)smem);
        else
            sweep_walk_block<R, UT, NS, DIR, MODE>(M, sm, it.a, it.b, E.seg);
    }
}

// ----------------------------------------------------------------------------- one launch per phase

// the register budgets of the single-grid kernels: cell state six blocks per SM (FP32
// bulk; five in the FP64 path), staged x sweep five
template <typename R, int NS>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 6 : 5) ens_cell_kernel(int mslot, const __grid_constant__ EnsDev E,
                                                       int stage) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Member sm;
    __shared__ int s_ok;
    // after a persistent sweep launch gave up, the stage states of this step were never
    // written: run nothing (the temperature warm start must not be overwritten)
    if (*(volatile int *)E.timeout) return;
    ens_cell_phase<R, NS>(M, E, stage, smem_raw, sm, s_ok);
}

template <typename R, typename UT, int NS, int MODE>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 5 : 3) ens_x_kernel(int mslot, const __grid_constant__ EnsDev E,
                                                    int stage) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Member sm;
    __shared__ int s_ok;
    ens_x_phase<R, UT, NS, MODE>(M, E, stage, smem_raw, sm, s_ok);
}

template <typename R, typename UT, int NS, int DIR, int MODE>
__global__ void __launch_bounds__(128) ens_walk_kernel(int mslot, const __grid_constant__ EnsDev E,
                                                       int stage) {
    const MechDev &M = c_mech[mslot];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Member sm;
    __shared__ int s_ok;
    ens_walk_phase<R, UT, NS, DIR, MODE>(M, E, stage, smem_raw, sm, s_ok);
}

template <typename R, int NS>
__global__ void __launch_bounds__(128) ens_final_kernel(const __grid_constant__ EnsDev E, int stage) {
    __shared__ Member sm;
    __shared__ int s_ok;
    if (*(volatile int *)E.timeout) return;     // a persistent sweep launch of this step gave up
    ens_final_phase<R, NS>(E, stage, sm, s_ok);
}

// Step prologue (run start): t from the caller, CFL, fixed dt, cleared maxima.
__global__ void ens_begin_kernel(const __grid_constant__ EnsDev E, const double *t_in, double cfl, double dt_fixed) {
    const int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= E.nmembers) return;
    const Member &m = E.tab[0][mi];
    m.clock[0] = t_in[mi];
    m.clock[2] = cfl;
    m.clock[3] = dt_fixed;
    m.rates[0] = m.rates[1] = m.rates[2] = 0ull;
}

__global__ void ens_dt_kernel(int mslot, const __grid_constant__ EnsDev E) {
    const MechDev &M = c_mech[mslot];
    const int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= E.nmembers) return;
    member_dt(M, E.tab[0][mi]);
}

// Step epilogue: advance the clock of members that did not fail, clear maxima.
__global__ void ens_end_kernel(const __grid_constant__ EnsDev E) {
    const int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= E.nmembers || *(volatile int *)E.timeout) return;
    const Member &m = E.tab[0][mi];
    if (*m.status == 0) m.clock[0] += m.clock[1];
    m.rates[0] = m.rates[1] = m.rates[2] = 0ull;
}

__global__ void ens_finish_kernel(const __grid_constant__ EnsDev E, double *t_out) {
    const int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= E.nmembers) return;
    t_out[mi] = E.tab[0][mi].clock[0];
}

// ----------------------------------------------------------------------------- persistent stage

// Grid-wide barrier of a cooperative launch with a bounded wait: after
// E.max_spins polls (~100 ns apart) it sets *E.timeout and returns false; the
// caller then leaves the kernel.  Arrivals are counted against E.bar_expect.
__device__ __forceinline__ bool grid_barrier(const EnsDev &E, int &s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = E.bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(E.bar, 1u) == E.bar_expect - 1) {
            atomicExch(E.bar, 0u);
            // every block is past its y items and none has taken a z item: restart both
            // work counters (the y one for the next launch)
            atomicExch(E.bar + 2, 0u);
            atomicExch(E.bar + 3, 0u);
            __threadfence();
            atomicAdd(E.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (*(volatile int *)E.timeout) {
                    ok = 0;
                    break;
                }
                if (++spins > E.max_spins) {
                    atomicExch(E.timeout, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_flag = ok;
    }
    __syncthreads();
    return s_flag != 0;
}

// The y and z sweeps of one RK stage of every member in one cooperative launch,
// separated by a grid barrier.  The stage's cell state and x sweep run before it, and
// in the FP32-bulk path the stage update after it, as work-list launches of their own
// (the x sweep's blocks fit three to an SM alone, two beside the walk's rings): the cell state is bound by FP64 latency and needs the 24 warps per SM that
// its own 80-register, 33 KB blocks give, which no launch that also holds the staged
// sweeps' registers and 75 KB rings can offer (a launch running every phase held the
// cell state at 8 warps per SM).
template <typename R, int NS>
__global__ void __launch_bounds__(128) ens_sweep_stage_kernel(int mslot, const __grid_constant__ EnsDev E,
                                                              int stage) {
    const MechDev &M = c_mech[mslot];
    using UT = typename std::conditional<sizeof(R) == 4, float, double>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Member sm;
    __shared__ int s_ok, s_flag, s_w;
    if (*(volatile int *)E.timeout) return;     // an earlier stage of this step gave up: run nothing
    ens_walk_phase_dynamic<R, UT, NS, 1, MODE_ACCUM>(M, E, stage, smem_raw, sm, s_ok, s_w);
    if (!grid_barrier(E, s_flag)) return;
    // FP32 bulk: the z sweep accumulates and an elementwise launch applies the stage (the
    // stage's FP64 operations would hold this launch's few warps); FP64: fused
    ens_walk_phase_dynamic<R, UT, NS, 2, sizeof(R) == 4 ? MODE_ACCUM : MODE_STAGE>(M, E, stage, smem_raw, sm, s_ok, s_w);
}

}  // namespace rf
