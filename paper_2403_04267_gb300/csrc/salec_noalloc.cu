// salec_noalloc.cu -- the Courant time step for callers that cannot allocate GPU memory.
//
// salec_step keeps its per-block minima in the caller's state buffer.  Some callers have
// no way to provide or allocate device memory for that: code running under an external
// memory manager that owns every device allocation, plug-ins that receive only the field
// pointers of someone else's simulation, or a process whose allocator is locked.  This
// entry point computes the same time step from caller-owned field buffers and keeps its
// scratch (the per-block minima, a completion counter and the result) in file-scope
// __device__ storage of fixed size, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "salec_internal.cuh"

namespace salec {

// Largest grid of 32 x 8-cell blocks the scratch holds: 65536 blocks, e.g. 4096 x 4096 cells.
constexpr int kNoAllocMaxBlocks = 65536;

// per-block minima of dx / (|v| + c)
static __device__ __align__(256) double g_noalloc_minima[kNoAllocMaxBlocks];

struct NoAllocControl {
    unsigned int counter;   // blocks finished; must be 0 when a launch starts
    int nan;                // a candidate was NaN; must be 0 when a launch starts
    double result;          // the time step of the last call
};
static __device__ __align__(256) NoAllocControl g_noalloc_control;

struct NoAllocArgs {
    int nr, nz, nmat;
    double dx, cfl, growth, dt_max, dt_prev;
    Mat mat[kMaxMat];
    const double2* fr[kMaxMat];
    const double* I;
    const double* D;
    const double2* v;
};

// The EoS, sound speed and candidate of the phase-0 kernel; per-block minima go to the
// file-scope scratch and the last block to finish reduces them.
__global__ void __launch_bounds__(kThreads) k_courant_noalloc(NoAllocArgs A, double* minima, NoAllocControl* ctl)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    double cand = INFINITY;
    if (i < A.nr && j < A.nz) {
        const int c = j * A.nr + i;
        double phi = 0.0, c2m = 0.0;
        const double Ic = A.I[c];
        for (int m = 0; m < A.nmat; ++m) {
            const double2 fr = A.fr[m][c];
            if (fr.x > 0.0) {
                double pm, c2;
                eos_eval(A.mat[m], fr.y, Ic, pm, c2);
                phi += fr.x;
                c2m = c2 > c2m ? c2 : c2m;
            }
        }
        if (phi > 0.0) {
            const int nv = A.nr + 1;
            const double2 va = A.v[j * nv + i], vb = A.v[j * nv + i + 1];
            const double2 vc = A.v[(j + 1) * nv + i + 1], vd = A.v[(j + 1) * nv + i];
            // the largest squared vertex speed by its bit pattern, as salec_step's first
            // kernel takes it: a NaN velocity is carried into the candidate, not dropped
            double w = va.x * va.x + va.y * va.y;
            w = max_nonneg(w, vb.x * vb.x + vb.y * vb.y);
            w = max_nonneg(w, vc.x * vc.x + vc.y * vc.y);
            w = max_nonneg(w, vd.x * vd.x + vd.y * vd.y);
            cand = A.dx / (sqrt(w) + sqrt(c2m));
            if (is_nan(cand)) atomicOr(&ctl->nan, 1);
        }
    }
    __shared__ double sh[kThreads / 32];
    __shared__ bool last;
    const int tid = threadIdx.y * kBlockX + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) cand = fmin(cand, __shfl_down_sync(0xffffffffu, cand, o));
    if ((tid & 31) == 0) sh[tid >> 5] = cand;
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y;
    if (tid == 0) {
        double b = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) b = fmin(b, sh[w]);
        minima[blockIdx.y * gridDim.x + blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(&ctl->counter, 1u) == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double m = INFINITY;
    for (int k = tid; k < nblk; k += kThreads) m = fmin(m, __ldcg(&minima[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) sh[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        double b = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) b = fmin(b, sh[w]);
        double dt = A.growth * A.dt_prev;
        const double cdt = A.cfl * b;
        dt = cdt < dt ? cdt : dt;
        dt = A.dt_max < dt ? A.dt_max : dt;
        ctl->result = dt;
        ctl->counter = 0u;
    }
}

namespace {

// Device addresses of the file-scope scratch, looked up once per device with that device
// current.  In host code the names g_noalloc_minima / g_noalloc_control are host-side
// stand-ins, not device addresses, so only these looked-up pointers go to the kernel.
// A device reset (cudaDeviceReset) ends the context they belong to: the call must not be
// used across one.
struct DeviceScratch {
    bool ready = false;
    double* minima = nullptr;
    NoAllocControl* control = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;
thread_local std::string g_noalloc_error;

salec_status noalloc_fail(salec_status st, const char* msg)
{
    g_noalloc_error = msg;
    return st;
}

}  // namespace

const char* noalloc_last_error() { return g_noalloc_error.c_str(); }

}  // namespace salec

using namespace salec;

extern "C" salec_status salec_courant_dt_noalloc(const salec_grid* grid, const salec_material* mats,
                                                 const double* const* fr, const double* I, const double* D,
                                                 const double* v, double dt_prev, double* dt_out, void* stream)
{
    (void)D;   // the sound speed does not depend on damage
    if (!grid) return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: null grid");
    if (grid->nr < 1 || grid->nz < 1 || grid->nmat < 1 || grid->nmat > kMaxMat || !(grid->dx > 0.0))
        return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: bad grid");
    const long long nbx = (grid->nr + kBlockX - 1) / kBlockX, nby = (grid->nz + kBlockY - 1) / kBlockY;
    if (nbx * nby > kNoAllocMaxBlocks)
        return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: grid larger than the fixed scratch "
                                          "(at most 65536 blocks of 32 x 8 cells, e.g. 4096 x 4096)");
    if (nby > 65535)    // the launch's largest grid height
        return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: more than 65535 rows of 8-cell blocks (nz > 524280)");
    if (!mats || !fr || !I || !v || !dt_out)
        return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: null argument");
    for (int m = 0; m < grid->nmat; ++m)
        if (!fr[m]) return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: null material field");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SALEC_EINVAL, "courant_dt_noalloc: device ordinal too large");
    DeviceScratch sc;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        DeviceScratch& d = g_scratch[dev];
        if (!d.ready) {
            void* pm = nullptr;
            void* pc = nullptr;
            e = cudaGetSymbolAddress(&pm, g_noalloc_minima);
            if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
            e = cudaGetSymbolAddress(&pc, g_noalloc_control);
            if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
            d.minima = static_cast<double*>(pm);
            d.control = static_cast<NoAllocControl*>(pc);
            d.ready = true;
        }
        sc = d;
    }
    NoAllocArgs A;
    A.nr = grid->nr; A.nz = grid->nz; A.nmat = grid->nmat;
    A.dx = grid->dx; A.cfl = grid->cfl; A.growth = grid->dt_growth; A.dt_max = grid->dt_max; A.dt_prev = dt_prev;
    for (int m = 0; m < kMaxMat; ++m) {
        A.fr[m] = m < grid->nmat ? reinterpret_cast<const double2*>(fr[m]) : nullptr;
        A.mat[m] = m < grid->nmat ? to_mat<double>(mats[m]) : Mat();
    }
    A.I = I;
    A.D = D;
    A.v = reinterpret_cast<const double2*>(v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counter and the NaN flag must start at zero; the scratch keeps whatever the
    // previous call left
    e = cudaMemsetAsync(sc.control, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
    k_courant_noalloc<<<dim3((unsigned)nbx, (unsigned)nby), dim3(kBlockX, kBlockY), 0, st>>>(A, sc.minima, sc.control);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
    NoAllocControl out;
    e = cudaMemcpyAsync(&out, sc.control, sizeof(NoAllocControl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(SALEC_ECUDA, cudaGetErrorString(e));
    // the failures salec_step reports in its status word: a NaN speed (bit 2) and a step
    // below dt_min (bit 4)
    if (out.nan) return noalloc_fail(SALEC_EUNSTABLE, "courant_dt_noalloc: NaN in the Courant candidates");
    if (out.result < grid->dt_min)
        return noalloc_fail(SALEC_EUNSTABLE, "courant_dt_noalloc: time step below dt_min");
    *dt_out = out.result;
    return SALEC_OK;
}
