// salec_persist.cu -- a batch of independent runs advanced by ONE persistent launch per
// chunk of steps: a cooperative grid of as many blocks as the device holds at once loops
// over the steps; in each step every block takes (run, tile) entries of the cell or vertex
// work list in turn for each of the six phases (the bodies of salec_phases.cuh, the same
// code per cell and vertex as the phase kernels), with a grid-wide barrier between phases
// and one pass of per-run Courant steps after phase 0.  It replaces the six launches and
// the Courant kernel of each batched step by barriers inside one kernel.
//
// The barrier is a counter and a generation word in device memory.  Every wait on it is
// bounded: after kGridWaitNs of %globaltimer a block records where it gave up, raises the
// error word (every other waiting block then leaves too) and the kernel returns; the host
// reads the word at its next poll and reports SALEC_ETIMEOUT.  A cooperative launch is
// refused unless every block is resident, so the barrier does not wait on blocks that
// cannot run.
#include <cuda_runtime.h>

#include "salec_phases.cuh"

namespace salec {

namespace {

constexpr unsigned long long kGridWaitNs = 2000000000ull;    // 2 s per barrier wait

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier: the writes of every block before it are seen by every block after
// it.  Thread 0 of each block arrives (after a fence that publishes its block's writes,
// ordered before it by the block barrier); the last to arrive resets the counter and
// advances the generation; the others wait for the new generation with an acquire load.
// Returns false when the wait ran out or another block raised the error word.
__device__ bool grid_sync(GridSync* gs, unsigned& gen, int where)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned target = gen + 1;
        int ok = 1;
        __threadfence();
        if (atomicAdd(&gs->arrive, 1u) == gridDim.x - 1) {
            atomicExch(&gs->arrive, 0u);
            __threadfence();
            atomicExch(&gs->gen, target);
            (void)ld_acquire(&gs->gen);     // acquire, as the waiting blocks do
        } else {
            const unsigned long long t0 = global_ns();
            unsigned spin = 0;
            while (ld_acquire(&gs->gen) != target) {
                if (*(volatile int*)&gs->err) { ok = 0; break; }
                if ((++spin & 255u) == 0 && global_ns() - t0 > kGridWaitNs) {
                    atomicCAS(&gs->where, 0, where);
                    atomicExch(&gs->err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        if (*(volatile int*)&gs->err) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    gen += 1;
    return s_ok != 0;
}

// Whether the block's run takes part in this phase, read once by thread 0 and shared, so
// the decision is the same for every thread of the block even while another block of the
// run sets its status word.
template <typename T>
__device__ __forceinline__ bool run_steps(const ParamsT<T>& P, bool phase0)
{
    bool go = false;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const DevScalars* s = P.p.scal;
        go = phase0 ? (s->t < s->t_end && s->status == 0) : s->active != 0;
    }
    return __syncthreads_or(go) != 0;
}

#define SALEC_PERSIST_PHASE(LIST, N, PHASE0, CALL)                                         \
    for (int k = blockIdx.x; k < (N); k += gridDim.x) {                                     \
        const BatchTile w = LIST[k];                                                        \
        const ParamsT<T>& P = runs[w.run];                                                  \
        if (run_steps<T>(P, PHASE0)) CALL(P, w.bx, w.by, w.g & 0xffff, w.g >> 16);          \
        __syncthreads();                                                                    \
    }

template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kPersistMaxThreads) kb_persistent(const ParamsT<T>* __restrict__ runs, int nruns,
                                                                    const BatchTile* __restrict__ cells, int ncells,
                                                                    const BatchTile* __restrict__ verts, int nverts,
                                                                    int steps, GridSync* gs)
{
    unsigned gen = 0;       // the generation word starts at 0 (cleared before the launch)
    const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int s = 0; s < steps; ++s) {
        const int where = 8 * s + 1;
        SALEC_PERSIST_PHASE(cells, ncells, true, (body_phase0<T, NM, STR, UNI>))
        if (!grid_sync(gs, gen, where)) return;
        // the Courant step of every run; a run at or past its end time or with a failure
        // status does nothing in this step
        for (int r = blockIdx.x * nthr + tid; r < nruns; r += gridDim.x * nthr) {
            const ParamsT<T>& P = runs[r];
            DevScalars* sc = P.p.scal;
            if (!(sc->t < sc->t_end) || sc->status != 0) {
                sc->active = 0;
                sc->maxbits = 0ull;
            } else {
                courant_dt<T>(P);
            }
        }
        if (!grid_sync(gs, gen, where + 1)) return;
        SALEC_PERSIST_PHASE(verts, nverts, false, (body_phase1<T, STR, UNI>))
        if (!grid_sync(gs, gen, where + 2)) return;
        SALEC_PERSIST_PHASE(cells, ncells, false, (body_phase2<T, NM, STR, UNI>))
        if (!grid_sync(gs, gen, where + 3)) return;
        SALEC_PERSIST_PHASE(cells, ncells, false, (body_phase3a<T, NM, STR, UNI>))
        if (!grid_sync(gs, gen, where + 4)) return;
        SALEC_PERSIST_PHASE(verts, nverts, false, (body_phase3b<T>))
        if (!grid_sync(gs, gen, where + 5)) return;
        SALEC_PERSIST_PHASE(cells, ncells, false, (body_phase3c<T, NM>))
        if (!grid_sync(gs, gen, where + 6)) return;
    }
}
#undef SALEC_PERSIST_PHASE

template <typename T, int NM, bool STR, bool UNI>
struct Persist {
    static void* fn() { return reinterpret_cast<void*>(kb_persistent<T, NM, STR, UNI>); }
};

template <typename T, typename Fn>
cudaError_t dispatch(int nmat, bool strength, bool uniform, Fn&& fn)
{
#define SALEC_PERSIST_CASE(NM_)                                                                      \
    case NM_:                                                                                         \
        if (uniform) return strength ? fn(Persist<T, NM_, true, true>()) : fn(Persist<T, NM_, false, true>()); \
        return strength ? fn(Persist<T, NM_, true, false>()) : fn(Persist<T, NM_, false, false>());
    switch (nmat) {
        SALEC_PERSIST_CASE(1)
        SALEC_PERSIST_CASE(2)
        SALEC_PERSIST_CASE(3)
    default: return cudaErrorInvalidValue;
    }
#undef SALEC_PERSIST_CASE
}

}  // namespace

// The resident grid of the persistent kernel for a block shape: every SM times the blocks
// of that shape it holds at once.
template <typename T>
cudaError_t prepare_batch_persistent(int nmat, bool strength, bool uniform, dim3 blk, int* ctas)
{
    if (blk.x * blk.y > (unsigned)kPersistMaxThreads) return cudaErrorInvalidConfiguration;
    return dispatch<T>(nmat, strength, uniform, [&](auto f) {
        const void* k = decltype(f)::fn();
        const size_t smem = phase3b_smem<T>(blk);
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)(blk.x * blk.y), smem);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) *ctas = sms * per_sm;
        return e;
    });
}

// `steps` batched steps of every run in one cooperative launch (the barrier words cleared
// first, on the same stream).  With expire, the arrival counter starts far above the grid
// size instead, so no block is ever the last to arrive at the first barrier: every wait
// there runs out (the test of the host's detection of that).
template <typename T>
cudaError_t launch_batch_persistent(const ParamsT<T>* runs, int nruns, int nmat, bool strength, bool uniform,
                                    const BatchTile* cells, int ncells, const BatchTile* verts, int nverts, dim3 blk,
                                    int ctas, int steps, GridSync* gs, bool expire, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GridSync), s);
    if (e == cudaSuccess && expire) e = cudaMemsetAsync(&gs->arrive, 0x40, sizeof(unsigned), s);   // 0x40404040
    if (e != cudaSuccess || steps < 1) return e;
    return dispatch<T>(nmat, strength, uniform, [&](auto f) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ctas);
        cfg.blockDim = blk;
        cfg.dynamicSmemBytes = phase3b_smem<T>(blk);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {(void*)&runs, (void*)&nruns, (void*)&cells, (void*)&ncells, (void*)&verts, (void*)&nverts,
                        (void*)&steps, (void*)&gs};
        return cudaLaunchKernelExC(&cfg, decltype(f)::fn(), args);
    });
}

template cudaError_t prepare_batch_persistent<double>(int, bool, bool, dim3, int*);
template cudaError_t prepare_batch_persistent<float>(int, bool, bool, dim3, int*);
template cudaError_t launch_batch_persistent<double>(const ParamsT<double>*, int, int, bool, bool, const BatchTile*, int,
                                                     const BatchTile*, int, dim3, int, int, GridSync*, bool, cudaStream_t);
template cudaError_t launch_batch_persistent<float>(const ParamsT<float>*, int, int, bool, bool, const BatchTile*, int,
                                                    const BatchTile*, int, dim3, int, int, GridSync*, bool, cudaStream_t);

}  // namespace salec
