// salec_kernels.cu -- the SALE cycle on sm_103a as one kernel per phase (bodies in
// salec_phases.cuh): single-run kernels over a grid of blocks, batched kernels over a work
// list of (run, tile) entries, and the read-out kernels.
#include <cuda_runtime.h>

#include "salec_phases.cuh"

namespace salec {


// ---------------------------------------------------------------------------------
// Kernels: single run (one grid of blocks over the run) and batched (one block per entry of
// a work list of (run, tile); a run's parameters are read from device memory; runs that
// reached their end time are skipped; each run keeps its own dt reduction).
// ---------------------------------------------------------------------------------

// The FP64 phase 0 (equation of state per material, artificial viscosity) holds more live
// values than 64 registers: with one resident block of the largest shape as its bound it
// takes 80-90 registers and spills nothing (under the default bound ptxas settled on 64
// and spilled 8-144 bytes a thread); the mixed form keeps the default.
template <typename T> struct Phase0Bound { static constexpr int min_blocks = sizeof(T) == 8 ? 1 : 0; };

template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads, Phase0Bound<T>::min_blocks) k_phase0(ParamsT<T> P) { body_phase0<T, NM, STR, UNI>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }
template <typename T>
__global__ void k_courant(ParamsT<T> P)
{
    if (threadIdx.x == 0) courant_dt<T>(P);
}

template <typename T>
cudaError_t launch_courant(const ParamsT<T>& P, cudaStream_t s)
{
    k_courant<T><<<1, 32, 0, s>>>(P);
    return cudaGetLastError();
}
template cudaError_t launch_courant<double>(const ParamsT<double>&, cudaStream_t);
template cudaError_t launch_courant<float>(const ParamsT<float>&, cudaStream_t);
template <typename T, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) k_phase1(ParamsT<T> P) { body_phase1<T, STR, UNI>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }
template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) k_phase2(ParamsT<T> P) { body_phase2<T, NM, STR, UNI>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }
template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) k_phase3a(ParamsT<T> P) { body_phase3a<T, NM, STR, UNI>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) k_phase3b(ParamsT<T> P) { body_phase3b<T>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }
template <typename T, int NM>
__global__ void __launch_bounds__(kMaxThreads) k_phase3c(ParamsT<T> P) { body_phase3c<T, NM>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y); }

// phase 0 decides for the whole step: a run at or past its end time, or one whose status
// reports a failure (non-positive volume or density, NaN, dt below dt_min), does nothing
template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads, Phase0Bound<T>::min_blocks) kb_phase0(const ParamsT<T>* __restrict__ runs,
                                                                                     const BatchTile* __restrict__ work)
{
    const BatchTile w = work[blockIdx.x];
    const ParamsT<T>& P = runs[w.run];
    const DevScalars* s = P.p.scal;
    if (!(s->t < s->t_end) || s->status != 0) return;
    body_phase0<T, NM, STR, UNI>(P, w.bx, w.by, w.g & 0xffff, w.g >> 16);
}
// the Courant step of every run; a run at or past its end time or with a failure status
// does nothing in this step (active = 0 tells the later kernels)
template <typename T>
__global__ void kb_courant(const ParamsT<T>* __restrict__ runs, int nruns)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    const ParamsT<T>& P = runs[r];
    DevScalars* s = P.p.scal;
    if (!(s->t < s->t_end) || s->status != 0) {
        s->active = 0;
        s->maxbits = 0ull;
        return;
    }
    courant_dt<T>(P);
}
#define SALEC_BATCHED(NAME, CALL)                                                          \
    {                                                                                      \
        const BatchTile w = work[blockIdx.x];                                              \
        const ParamsT<T>& P = runs[w.run];                                                 \
        if (P.p.scal->active == 0) return;                                                 \
        CALL(P, w.bx, w.by, w.g & 0xffff, w.g >> 16);                                      \
    }
template <typename T, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) kb_phase1(const ParamsT<T>* __restrict__ runs, const BatchTile* __restrict__ work)
SALEC_BATCHED(phase1, (body_phase1<T, STR, UNI>))
template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) kb_phase2(const ParamsT<T>* __restrict__ runs, const BatchTile* __restrict__ work)
SALEC_BATCHED(phase2, (body_phase2<T, NM, STR, UNI>))
template <typename T, int NM, bool STR, bool UNI>
__global__ void __launch_bounds__(kMaxThreads) kb_phase3a(const ParamsT<T>* __restrict__ runs, const BatchTile* __restrict__ work)
SALEC_BATCHED(phase3a, (body_phase3a<T, NM, STR, UNI>))
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) kb_phase3b(const ParamsT<T>* __restrict__ runs, const BatchTile* __restrict__ work)
SALEC_BATCHED(phase3b, (body_phase3b<T>))
template <typename T, int NM>
__global__ void __launch_bounds__(kMaxThreads) kb_phase3c(const ParamsT<T>* __restrict__ runs, const BatchTile* __restrict__ work)
SALEC_BATCHED(phase3c, (body_phase3c<T, NM>))

// The mixed form's remap kernels for one hydrodynamic material (and its vertex remap for
// any material count, single and batched) are latency-bound (19-34 % of DRAM peak at
// 62-75 % occupancy): their registers are capped so that a full SM of threads (4 blocks
// of the largest shape) fits, at the cost of a few bytes of spill.  With more materials
// or strength the cell remap would spill heavily under such a cap; the FP64 kernels are
// bound by the FP64 pipe.  Both keep the compiler's own register choice.
template <>
__global__ void __launch_bounds__(kMaxThreads, 4) k_phase3a<float, 1, false, true>(ParamsT<float> P)
{
    body_phase3a<float, 1, false, true>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}
template <>
__global__ void __launch_bounds__(kMaxThreads, 4) k_phase3a<float, 1, false, false>(ParamsT<float> P)
{
    body_phase3a<float, 1, false, false>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}
template <>
__global__ void __launch_bounds__(kMaxThreads, 4) k_phase3b<float>(ParamsT<float> P)
{
    body_phase3b<float>(P, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}
template <>
__global__ void __launch_bounds__(kMaxThreads, 4) kb_phase3b<float>(const ParamsT<float>* __restrict__ runs,
                                                                   const BatchTile* __restrict__ work)
{
    const BatchTile w = work[blockIdx.x];
    const ParamsT<float>& P = runs[w.run];
    if (P.p.scal->active == 0) return;
    body_phase3b<float>(P, w.bx, w.by, w.g & 0xffff, w.g >> 16);
}

// ---------------------------------------------------------------------------------
// Read-out kernels
// ---------------------------------------------------------------------------------
template <typename T, int NM>
__global__ void __launch_bounds__(kMaxThreads) k_pressure(ParamsT<T> P, double* out)
{
    typedef VT<T> V;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= P.nr || j >= P.nz) return;
    const int c = j * P.nr + i;
    const PtrsT<T>& p = P.p;
    const T D = P.any_strength ? p.s2d[c].y : T(0);
    T phat = T(0), phi = T(0);
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const typename V::T2 fr = p.fr[m][c];
        if (fr.x > T(0)) {
            T pm, c2;
            eos_eval<T>(P.mat[m], fr.y, T(p.I[c]), pm, c2);
            const T pmin = (T(1) - D) * P.mat[m].p_t * expansion_weight(P.mat[m], fr.y);
            pm = pm < pmin ? pmin : pm;
            phat += fr.x * pm;
            phi += fr.x;
        }
    }
    out[c] = phi > T(0) ? double(phat / phi) : 0.0;
}

// one thread per column: scan down from the top for sum_m f_m >= 1/2
template <typename T, int NM>
__global__ void k_column_heights(ParamsT<T> P, double* h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nr) return;
    const int nr = P.nr, nz = P.nz;
    auto phi_at = [&](int j) {
        double f = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) f += double(P.p.fr[m][j * nr + i].x);
        return f;
    };
    double out = 0.0;
    double up = 0.0;
    for (int j = nz - 1; j >= 0; --j) {
        const double phi = phi_at(j);
        if (phi >= 0.5) {
            const double zc = P.p.zc[j];
            out = (j == nz - 1) ? zc : zc + (phi - 0.5) / (phi - up) * (P.p.zc[j + 1] - zc);
            break;
        }
        up = phi;
    }
    h[i] = out;
}

// per-block FP64 sums of mass, z-momentum, kinetic and internal energy
template <typename T, int NM>
__global__ void __launch_bounds__(kMaxThreads) k_conservation(ParamsT<T> P, double* partial4)
{
    typedef VT<T> V;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    const PtrsT<T>& p = P.p;
    auto cmass = [&](int ci, int cj) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const typename V::T2 fr = p.fr[m][cj * nr + ci];
            s += double(fr.x) * double(fr.y);
        }
        return s * double(p.A_Z[ci] * p.dz[cj]);
    };
    double mass = 0.0, ie = 0.0, pz = 0.0, ke = 0.0;
    if (i < nr && j < nz) {
        const double M = cmass(i, j);
        mass = M;
        ie = M * p.I[j * nr + i];
    }
    if (i <= nr && j <= nz) {
        double m = 0.0;
        for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di) {
                const int ci = i + di, cj = j + dj;
                if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                m += 0.25 * cmass(ci, cj);
            }
        const typename V::T2 vv = p.v[j * (nr + 1) + i];
        pz = m * double(vv.y);
        ke = 0.5 * m * (double(vv.x) * double(vv.x) + double(vv.y) * double(vv.y));
    }
    __shared__ double sh[kMaxThreads / 32];
    const double a = block_sum(mass, sh), b = block_sum(pz, sh), c = block_sum(ke, sh), d = block_sum(ie, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        partial4[4 * blk + 0] = a;
        partial4[4 * blk + 1] = b;
        partial4[4 * blk + 2] = c;
        partial4[4 * blk + 3] = d;
    }
}

// ---------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------
static dim3 grid_of(int ni, int nj, dim3 blk) { return dim3((ni + blk.x - 1) / blk.x, (nj + blk.y - 1) / blk.y); }
static dim3 cell_grid(int nr, int nz) { return grid_of(nr, nz, dim3(kBlockX, kBlockY)); }
static dim3 vert_grid(int nr, int nz) { return grid_of(nr + 1, nz + 1, dim3(kBlockX, kBlockY)); }

int cell_blocks(int nr, int nz) { dim3 g = cell_grid(nr, nz); return (int)(g.x * g.y); }
int vertex_blocks(int nr, int nz) { dim3 g = vert_grid(nr, nz); return (int)(g.x * g.y); }
int launches_per_step() { return 6; }
int kernels_per_step() { return 7; }     // the six phases and the Courant kernel
// kernels 1 (forces) and 4 (momentum remap) run over vertices, the others over cells
bool kernel_on_vertices(int k) { return k == 1 || k == 4; }
int tiles_of(int nr, int nz, int k, dim3 blk)
{
    const dim3 g = kernel_on_vertices(k) ? grid_of(nr + 1, nz + 1, blk) : grid_of(nr, nz, blk);
    return (int)(g.x * g.y);
}

const char* kernel_name(int k)
{
    static const char* names[] = {"k_phase0", "k_phase1", "k_phase2", "k_phase3a", "k_phase3b", "k_phase3c"};
    return (k >= 0 && k < 6) ? names[k] : "";
}

// One cycle with per-kernel block shapes; with ev != nullptr an event is recorded before the
// first kernel and after each kernel (7 events) for per-kernel durations.
template <typename T, int NM, bool STR, bool UNI>
static cudaError_t step_impl(const ParamsT<T>& P, const dim3* blk, cudaStream_t s, cudaEvent_t* ev)
{
    const int nr = P.nr, nz = P.nz;
    if (ev) cudaEventRecord(ev[0], s);
    k_phase0<T, NM, STR, UNI><<<grid_of(nr, nz, blk[0]), blk[0], 0, s>>>(P);
    k_courant<T><<<1, 32, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[1], s);
    k_phase1<T, STR, UNI><<<grid_of(nr + 1, nz + 1, blk[1]), blk[1], 0, s>>>(P);
    if (ev) cudaEventRecord(ev[2], s);
    k_phase2<T, NM, STR, UNI><<<grid_of(nr, nz, blk[2]), blk[2], 0, s>>>(P);
    if (ev) cudaEventRecord(ev[3], s);
    k_phase3a<T, NM, STR, UNI><<<grid_of(nr, nz, blk[3]), blk[3], 0, s>>>(P);
    if (ev) cudaEventRecord(ev[4], s);
    k_phase3b<T><<<grid_of(nr + 1, nz + 1, blk[4]), blk[4], phase3b_smem<T>(blk[4]), s>>>(P);
    if (ev) cudaEventRecord(ev[5], s);
    k_phase3c<T, NM><<<grid_of(nr, nz, blk[5]), blk[5], 0, s>>>(P);
    if (ev) cudaEventRecord(ev[6], s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const ParamsT<T>& P, const dim3* blk, cudaStream_t s, cudaEvent_t* ev)
{
    const bool st = P.any_strength != 0;
    if (P.uniform) {
        switch (P.nmat) {
        case 1: return st ? step_impl<T, 1, true, true>(P, blk, s, ev) : step_impl<T, 1, false, true>(P, blk, s, ev);
        case 2: return st ? step_impl<T, 2, true, true>(P, blk, s, ev) : step_impl<T, 2, false, true>(P, blk, s, ev);
        case 3: return st ? step_impl<T, 3, true, true>(P, blk, s, ev) : step_impl<T, 3, false, true>(P, blk, s, ev);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (P.nmat) {
    case 1: return st ? step_impl<T, 1, true, false>(P, blk, s, ev) : step_impl<T, 1, false, false>(P, blk, s, ev);
    case 2: return st ? step_impl<T, 2, true, false>(P, blk, s, ev) : step_impl<T, 2, false, false>(P, blk, s, ev);
    case 3: return st ? step_impl<T, 3, true, false>(P, blk, s, ev) : step_impl<T, 3, false, false>(P, blk, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

// One cycle of every run of a batch: work[k] lists the (run, tile) entries of kernel k
// (ntiles[k] of them) for block shape blk[k].
template <typename T, int NM, bool STR, bool UNI>
static cudaError_t batch_impl(const ParamsT<T>* runs, int nruns, const BatchTile* const* work, const int* ntiles,
                              const dim3* blk, cudaStream_t s, cudaEvent_t* ev)
{
    if (ev) cudaEventRecord(ev[0], s);
    kb_phase0<T, NM, STR, UNI><<<ntiles[0], blk[0], 0, s>>>(runs, work[0]);
    kb_courant<T><<<(nruns + 127) / 128, 128, 0, s>>>(runs, nruns);
    if (ev) cudaEventRecord(ev[1], s);
    kb_phase1<T, STR, UNI><<<ntiles[1], blk[1], 0, s>>>(runs, work[1]);
    if (ev) cudaEventRecord(ev[2], s);
    kb_phase2<T, NM, STR, UNI><<<ntiles[2], blk[2], 0, s>>>(runs, work[2]);
    if (ev) cudaEventRecord(ev[3], s);
    kb_phase3a<T, NM, STR, UNI><<<ntiles[3], blk[3], 0, s>>>(runs, work[3]);
    if (ev) cudaEventRecord(ev[4], s);
    kb_phase3b<T><<<ntiles[4], blk[4], phase3b_smem<T>(blk[4]), s>>>(runs, work[4]);
    if (ev) cudaEventRecord(ev[5], s);
    kb_phase3c<T, NM><<<ntiles[5], blk[5], 0, s>>>(runs, work[5]);
    if (ev) cudaEventRecord(ev[6], s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_step(const ParamsT<T>* runs_dev, int nruns, int nmat, bool strength, bool uniform, const BatchTile* const* work,
                              const int* ntiles, const dim3* blk, cudaStream_t s, cudaEvent_t* ev)
{
    // every run of the batch on a uniform grid: the uniform form
    if (uniform) {
        switch (nmat) {
        case 1: return strength ? batch_impl<T, 1, true, true>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 1, false, true>(runs_dev, nruns, work, ntiles, blk, s, ev);
        case 2: return strength ? batch_impl<T, 2, true, true>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 2, false, true>(runs_dev, nruns, work, ntiles, blk, s, ev);
        case 3: return strength ? batch_impl<T, 3, true, true>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 3, false, true>(runs_dev, nruns, work, ntiles, blk, s, ev);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (nmat) {
    case 1: return strength ? batch_impl<T, 1, true, false>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 1, false, false>(runs_dev, nruns, work, ntiles, blk, s, ev);
    case 2: return strength ? batch_impl<T, 2, true, false>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 2, false, false>(runs_dev, nruns, work, ntiles, blk, s, ev);
    case 3: return strength ? batch_impl<T, 3, true, false>(runs_dev, nruns, work, ntiles, blk, s, ev) : batch_impl<T, 3, false, false>(runs_dev, nruns, work, ntiles, blk, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_pressure(const ParamsT<T>& P, double* out, cudaStream_t s)
{
    const dim3 blk(kBlockX, kBlockY), g = cell_grid(P.nr, P.nz);
    switch (P.nmat) {
    case 1: k_pressure<T, 1><<<g, blk, 0, s>>>(P, out); break;
    case 2: k_pressure<T, 2><<<g, blk, 0, s>>>(P, out); break;
    case 3: k_pressure<T, 3><<<g, blk, 0, s>>>(P, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_column_heights(const ParamsT<T>& P, double* h, cudaStream_t s)
{
    const int t = 128, b = (P.nr + t - 1) / t;
    switch (P.nmat) {
    case 1: k_column_heights<T, 1><<<b, t, 0, s>>>(P, h); break;
    case 2: k_column_heights<T, 2><<<b, t, 0, s>>>(P, h); break;
    case 3: k_column_heights<T, 3><<<b, t, 0, s>>>(P, h); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_conservation(const ParamsT<T>& P, double* partial4, int* nblocks, cudaStream_t s)
{
    const dim3 blk(kBlockX, kBlockY), g = vert_grid(P.nr, P.nz);
    *nblocks = (int)(g.x * g.y);
    switch (P.nmat) {
    case 1: k_conservation<T, 1><<<g, blk, 0, s>>>(P, partial4); break;
    case 2: k_conservation<T, 2><<<g, blk, 0, s>>>(P, partial4); break;
    case 3: k_conservation<T, 3><<<g, blk, 0, s>>>(P, partial4); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Per-run scalars of a batch gathered into one array (t, dt, step count, status, t_end).
template <typename T>
__global__ void k_batch_poll(const ParamsT<T>* __restrict__ runs, int n, double* out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const DevScalars* s = runs[r].p.scal;
    out[5 * r + 0] = s->t;
    out[5 * r + 1] = s->dt;
    out[5 * r + 2] = (double)s->nstep;
    out[5 * r + 3] = (double)s->status;
    out[5 * r + 4] = s->t_end;
}

template <typename T>
cudaError_t launch_batch_poll(const ParamsT<T>* runs_dev, int n, double* out, cudaStream_t s)
{
    k_batch_poll<T><<<(n + 127) / 128, 128, 0, s>>>(runs_dev, n, out);
    return cudaGetLastError();
}
template cudaError_t launch_batch_poll<double>(const ParamsT<double>*, int, double*, cudaStream_t);
template cudaError_t launch_batch_poll<float>(const ParamsT<float>*, int, double*, cudaStream_t);

template cudaError_t launch_step<double>(const ParamsT<double>&, const dim3*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_step<float>(const ParamsT<float>&, const dim3*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_batch_step<double>(const ParamsT<double>*, int, int, bool, bool, const BatchTile* const*, const int*,
                                               const dim3*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_batch_step<float>(const ParamsT<float>*, int, int, bool, bool, const BatchTile* const*, const int*,
                                              const dim3*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_pressure<double>(const ParamsT<double>&, double*, cudaStream_t);
template cudaError_t launch_pressure<float>(const ParamsT<float>&, double*, cudaStream_t);
template cudaError_t launch_column_heights<double>(const ParamsT<double>&, double*, cudaStream_t);
template cudaError_t launch_column_heights<float>(const ParamsT<float>&, double*, cudaStream_t);
template cudaError_t launch_conservation<double>(const ParamsT<double>&, double*, int*, cudaStream_t);
template cudaError_t launch_conservation<float>(const ParamsT<float>&, double*, int*, cudaStream_t);

}  // namespace salec
