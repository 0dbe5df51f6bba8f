// Batched persistent step: many independent runs of uneven ion count advance one
// step in ONE kernel launch (replayed from a CUDA graph).
//
// Every run's step is split into tasks of its four phases (scan tiles of 128 ions,
// pair units of one target tile x one source chunk, kick tiles, one grain-tail task).
// A persistent grid of at most the resident number of CTAs takes tasks from a global
// counter in phase-major order (all scan tiles, then all pair units, then all kick
// tiles, then all grain tails; runs in order inside each phase).  A task of phase p of
// run r first waits until run r's phase p-1 counter reaches its target; every task it
// waits for was handed out earlier to a CTA that is running, so the waits end (and
// each is bounded anyway: it gives up after spin_limit polls and sets an error).
// The counters only grow (target = (batch step + 1) x tasks per phase), so nothing
// is reset between launches; the last CTA to leave advances the batch step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "od_device.cuh"

namespace od {

constexpr int BATCH_BT = BATCH_TILE;

__device__ __forceinline__ unsigned long long ld_acquire_u64c(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// phase_end: cumulative task-index ends of phases 0..3.  tune = 1: a tuning launch whose
// task list holds only pair units and kick tiles; the pair units do not wait, the kick
// tiles wait for their run's pair units as in a step (on the tuning launch's own counters)
// and evaluate accelerations only (kick mode 1: no velocity update, no collisions), so the
// runs' states are not changed.
// held to 128 registers: four CTAs of 128 per SM
template <int IPT>
__global__ void __launch_bounds__(BATCH_BT, 65536 / (BATCH_BT * 128))
    k_batch_step(const RunDesc* __restrict__ runs, const int2* __restrict__ tasks, int4 phase_end, long long T,
                 BatchCtrl* bc, unsigned long long* done, int R, long long spin_limit, int tune)
{
    __shared__ float4 sj[BATCH_BT];
    __shared__ float s_acc[2][3][BATCH_BT / 32][SYM_SUB];
    __shared__ long long s_task;
    __shared__ int s_timeout;
    const unsigned long long bstep = bc->step;
    // every launch draws exactly T + gridDim.x tickets (T tasks plus one failing draw per CTA)
    const unsigned long long base = bstep * (unsigned long long)(T + gridDim.x);
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = (long long)(atomicAdd(&bc->task_next, 1ull) - base);
        __syncthreads();
        const long long t = s_task;
        if (t >= T) break;
        const int2 tk = tasks[t];
        const RunDesc& d = runs[tk.x];
        const int phase = t < phase_end.x ? 0 : t < phase_end.y ? 1 : t < phase_end.z ? 2 : 3;
        if (phase > 1 || (phase == 1 && !tune)) {
            // wait for the previous phase of this run
            if (threadIdx.x == 0) {
                const unsigned long long per = phase == 1 ? (unsigned long long)d.nA
                                                          : phase == 2 ? (unsigned long long)d.F.U
                                                                       : (unsigned long long)d.nK;
                const unsigned long long target = (bstep + 1) * per;
                const unsigned long long* cnt = done + (long long)(phase - 1) * R + tk.x;
                long long spins = 0;
                unsigned ns = 64;
                s_timeout = 0;
                while (ld_acquire_u64c(cnt) < target) {
                    if (++spins > spin_limit) {
                        s_timeout = 1;
                        atomicOr(&bc->err, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 2048) ns *= 2;
                }
            }
            __syncthreads();
        }
        switch (phase) {
        case 0: push_scan_body<BATCH_BT>(d.P, d.B, d.nA, 1.4426950408889634 * d.P.lam_inv, tk.y); break;
        case 1:
            if (d.F.sym) {
                int I, J;
                tri_unit(tk.y, d.F.JS, I, J);
                sym2_unit<BATCH_BT, IPT>(d.B.fpos, d.F, I, J, s_acc, sj);
            } else {
                forces_unit<BATCH_BT, IPT>(d.B.fpos, d.B.part, d.F, tk.y / d.F.JS, tk.y % d.F.JS, sj);
            }
            break;
        case 2: kick_body<BATCH_BT, 1>(d.P, d.B, d.F, tune ? 1 : 0, tk.y); break;
        default: dust_body<false>(d.P, d.B, d.nK, 0); break;
        }
        // publish completion of this task to the run's phase counter
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && phase < 3) atomicAdd(done + (long long)phase * R + tk.x, 1ull);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bc->exit_count, 1u) == gridDim.x - 1) {
            bc->exit_count = 0u;
            bc->step = bstep + 1;
        }
    }
}

static void* batch_fn(int ipt)
{
    switch (ipt) {
    case 2: return (void*)k_batch_step<2>;
    case 4: return (void*)k_batch_step<4>;
    default: return (void*)k_batch_step<8>;
    }
}

int batch_blocks_per_sm(int ipt)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_fn(ipt), BATCH_BT, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

int launch_batch(int ipt, int grid, const RunDesc* runs, const int2* tasks, int4 phase_end, long long T,
                 BatchCtrl* bc, unsigned long long* done, int R, long long spin_limit, int tune, cudaStream_t s)
{
    switch (ipt) {
    case 2:
        k_batch_step<2><<<grid, BATCH_BT, 0, s>>>(runs, tasks, phase_end, T, bc, done, R, spin_limit, tune);
        break;
    case 4:
        k_batch_step<4><<<grid, BATCH_BT, 0, s>>>(runs, tasks, phase_end, T, bc, done, R, spin_limit, tune);
        break;
    default:
        k_batch_step<8><<<grid, BATCH_BT, 0, s>>>(runs, tasks, phase_end, T, bc, done, R, spin_limit, tune);
        break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

// the pair partition of one run inside a batch: tiles of BATCH_BT * ipt targets, source
// chunks of jc, every unit its own task (G = U, slot = chunk); jc = 0 selects the
// symmetric tile pairs of the packed kernel
ForceArgs batch_plan(int N, int ipt, int jc)
{
    ForceArgs F{};
    F.TI = BATCH_BT * ipt;
    F.n_pad = N == 0 ? 0 : (N + F.TI - 1) / F.TI * F.TI;
    if (F.n_pad == 0) return F;
    if (jc == 0) {
        // symmetric tile pairs (I, J >= I) into the fixed-point accumulators
        const int T = F.n_pad / F.TI;
        F.sym = 1;
        F.JC = F.TI;
        F.JS = T;
        F.W = 0;
        F.U = (long long)T * (T + 1) / 2;
        F.G = (int)F.U;
        return F;
    }
    F.JC = std::max(BATCH_BT, std::min(jc, F.n_pad) / BATCH_BT * BATCH_BT);
    F.JS = (F.n_pad + F.JC - 1) / F.JC;
    F.U = (long long)(F.n_pad / F.TI) * F.JS;
    F.G = (int)F.U;
    F.W = F.JS;
    return F;
}

}  // namespace od
