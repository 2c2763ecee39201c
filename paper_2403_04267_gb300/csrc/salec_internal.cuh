// salec_internal.cuh -- shared definitions of the CUDA library: parameter blocks passed
// to the kernels by value, the device-state layout, and the material laws used on both
// the host (set-up) and the device (time step).
//
// Two arithmetic forms share the kernels through the element type T:
//   T = double  the FP64 form;
//   T = float   the mixed form: fields, stencils and material laws in FP32, while the
//               specific internal energy I, its updates, the Courant reduction and the
//               conservation sums stay FP64.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/salec.h"

namespace salec {

constexpr int kMaxMat = 3;
constexpr int kBlockX = 32;
constexpr int kBlockY = 8;
constexpr int kThreads = kBlockX * kBlockY;
constexpr int kMaxThreads = 512;      // largest block shape any kernel is launched with

// one entry of a batched launch: block (bx, by) of run `run`, whose grid of blocks is
// (g & 0xffff) x (g >> 16)
struct BatchTile { int run, bx, by, g; };

// Grid-wide barrier of the persistent batched kernel: arrival counter, generation, error
// word (a wait ran out) and where it ran out (8 x step + barrier index + 1).
struct GridSync { unsigned arrive, gen; int err, where; };
constexpr int kPersistMaxThreads = 256;     // largest block of the persistent batched kernel

// vector types of an element type
template <typename T> struct VT;
template <> struct VT<double> {
    typedef double2 T2;
    typedef double4_32a T4;
    __host__ __device__ static double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct VT<float> {
    typedef float2 T2;
    typedef float4 T4;
    __host__ __device__ static float2 mk(float a, float b) { return make_float2(a, b); }
};

// Material constants with the derived quantities the kernels use.
template <typename T>
struct MatT {
    int eos, strength;
    T rho0, inv_rho0, rho0sq_E0, A, B, E0, a, b, alpha, beta, Eiv, Ecv, inv_dE, gamma;
    T Yi0, mui, Yim, Yd0, mud, Ydm, inv_Yspan, G, eps_fb, B_dam, p_bd, p_t, c2_floor;
    T rho_f, inv_rho_f;     // the Tillotson density floor 1e-12 rho0 and its reciprocal
};
typedef MatT<double> Mat;

// The fused step's queue of tiles that need the whole cycle: filled by the rest-tile
// kernel (count), drained by the persistent tile kernel (next).
struct TileWork {
    int count;      // queued tiles at the front of the list: tiles that took the whole cycle
                    // in the step before (their cycles are the longest)
    int next;       // queued tiles handed out
    int back;       // queued tiles at the back of the list: tiles queued for a neighbour
    int copy_next;  // groups of 32 tiles handed to the copy kernel that runs beside the tile kernel
};

// Scalars of a run, resident on the device.
struct DevScalars {
    double t, dt, dt_prev, t_end;   // t_end: a batched run stops stepping once t >= t_end
    double mass_out, mass_discarded, mass_pml, zmom_out;
    unsigned long long nstep;
    unsigned long long maxbits;   // running max of the blocks' Courant rates (FP64 bit patterns)
    int status;             // bit 1: non-positive volume or density, 2: NaN, 4: dt < dt_min
    int active;             // the run stepped in the current batched step
    float dtf;              // dt rounded to FP32 (the mixed form's kernels read it without a conversion)
};

// Device pointers into the caller's state buffer.
template <typename T>
struct PtrsT {
    typedef typename VT<T>::T2 T2;
    typedef typename VT<T>::T4 T4;
    // persistent cell state
    T2* fr[kMaxMat];        // (f_m, rho_m)
    double* I;              // specific internal energy (FP64 in every form)
    T2* s01;                // (s_rr, s_zz)        [strength only]
    T2* s2d;                // (s_rz, D)           [strength only]
    T* pmax;                // running peak over-pressure
    T2* v;                  // vertex (v_r, v_z)
    // PML auxiliaries (compact strips)
    T2* pb_c;               // bottom cells (phi1, phi3), index j*nr + i, j < pb
    T* pb_psi2;             // bottom cells psi2
    T4* pb_v;               // bottom vertices (phi2r, phi2z, psi1r, psi1z), index j*(nr+1)+i, j < pb
    T2* pr_c;               // right cells (phi1, phi3), index j*pr + (i - (nr - pr))
    T* pr_psi2;
    T4* pr_v;               // right vertices, index j*pr + (i - (nr - pr + 1)), i > nr - pr
    // geometry (per radian): the radial face at r_i of row j has area rR[i] dz[j], the
    // vertical faces of column i area A_Z[i], cell (i,j) volume A_Z[i] dz[j]
    const T* rR;            // nr+1 vertex radii r_i
    const T* rc;            // nr   cell-centre radii
    const T* A_Z;           // nr   vertical face areas r_c dr
    const T* invAZ;         // nr   1 / A_Z
    const T* inv2rc;        // nr   1 / (2 r_c)
    const T* dr;            // nr   column widths
    const T* idr;           // nr   1 / dr
    const T* dz;            // nz   row heights
    const T* idz;           // nz   1 / dz
    const double* zc;       // nz   cell-centre heights (read-outs)
    // the same for a uniform grid of dx cells, one entry per column for every row
    const T* A_R;           // nr+1 radial face areas r_i dx
    const T* V;             // nr   cell volumes r_c dx^2
    const T* invV;          // nr   1 / V
    const T* p0;            // nz reference pressure per row
    const T* rho_ref;       // nz
    const double* I_ref;    // nz
    const T* dB_c;          // nz   bottom-strip profile at cell centres
    const T* dB_v;          // nz+1 bottom-strip profile at vertices
    const T* dR_c;          // nr
    const T* dR_v;          // nr+1
    // per-step scratch
    T2* PM;                 // (P, M) per cell
    T2* pbphi;              // (p_bar, Phi) per cell
    T2* vL;                 // Lagrangian vertex velocity
    T* mv;                  // vertex mass
    T* dK;                  // Lagrangian kinetic-energy deficit per vertex
    T* kheat;               // specific heat returned per vertex
    T2* frL[kMaxMat];       // Lagrangian (f_m^L, rho_m^L)
    T* VL;                  // Lagrangian cell volume
    double* IL;             // Lagrangian specific internal energy
    T2* sL01;               // Lagrangian (s_rr, s_zz)
    T2* sL2d;               // Lagrangian (s_rz, D)
    T* dMR;                 // signed mass flux through radial faces, (nr+1) x nz
    T* dMZ;                 // signed mass flux through vertical faces, nr x (nz+1)
    T2* eosc;               // fused form: each cell's equation of state at the current state,
                            // (p_m after the tension cut-off, c^2) for one material,
                            // (p_hat = sum f_m p_m, max c_m^2) for several
    double* partial;        // per-block reduction partials
    DevScalars* scal;
};

// Where a fused step writes the fields it rewrites (the other copy of the ping-pong pair;
// the kernel reads the current copy through ParamsT::p).
template <typename T>
struct OutPtrsT {
    typedef typename VT<T>::T2 T2;
    typedef typename VT<T>::T4 T4;
    T2* fr[kMaxMat];
    double* I;
    T2* s01;
    T2* s2d;
    T2* v;
    T2* pb_c;
    T* pb_psi2;
    T4* pb_v;
    T2* pr_c;
    T* pr_psi2;
    T4* pr_v;
    T2* eosc;
    // tiles at rest: rest_in[t] = 1 when the step that wrote the copy read here took tile t
    // through the quiescent path (its outputs are then its inputs); this step writes
    // rest_out.  work counts and hands out the tiles this step runs through the whole
    // cycle (list: their indices); work_next is zeroed for the next step.
    const unsigned char* rest_in;
    unsigned char* rest_out;
    TileWork* work;
    TileWork* work_next;
    int* list;
    int ctas;               // CTAs of the persistent tile kernel (all the device holds at once)
};

template <typename T>
struct ParamsT {
    int nr, nz, nmat, pr, pb, bc_top, bc_bottom, any_strength, nblk_cells;
    int uniform;            // every cell dx square: the kernels' uniform-grid form
    T cfl, g, cq, cl, f_min;
    T dx, dx2, idx;         // uniform grid: cell size, its square and inverse
    double dxd, cfld, growth, dt_max, dt_min;
    T alpha_b, alpha_r;     // relaxation rates of the bottom / right strips' auxiliaries (1/s)
    MatT<T> mat[kMaxMat];
    PtrsT<T> p;
};

// The material constants of the public struct with the derived quantities, in T.
template <typename T>
inline MatT<T> to_mat(const salec_material& s)
{
    MatT<T> m;
    memset(&m, 0, sizeof(m));
    m.eos = s.eos; m.strength = s.strength;
    m.rho0 = T(s.rho0); m.inv_rho0 = T(1.0 / s.rho0);
    m.rho0sq_E0 = T(s.eos == SALEC_EOS_TILLOTSON ? s.rho0 * s.rho0 / s.E0 : 0.0);
    m.A = T(s.A); m.B = T(s.B); m.E0 = T(s.E0); m.a = T(s.a); m.b = T(s.b); m.alpha = T(s.alpha);
    m.beta = T(s.beta); m.Eiv = T(s.Eiv); m.Ecv = T(s.Ecv);
    m.inv_dE = T((s.Ecv > s.Eiv) ? 1.0 / (s.Ecv - s.Eiv) : 0.0);
    m.gamma = T(s.gamma);
    m.Yi0 = T(s.Yi0); m.mui = T(s.mui); m.Yim = T(s.Yim); m.Yd0 = T(s.Yd0); m.mud = T(s.mud); m.Ydm = T(s.Ydm);
    m.inv_Yspan = T((s.Yim != s.Yi0) ? 1.0 / (s.Yim - s.Yi0) : 0.0);
    m.G = T(s.strength == SALEC_STRENGTH_COLLINS ? s.G : 0.0);
    m.eps_fb = T(s.eps_fb); m.B_dam = T(s.B_dam); m.p_bd = T(s.p_bd); m.p_t = T(s.p_t);
    m.c2_floor = T(s.eos == SALEC_EOS_TILLOTSON ? 0.01 * s.A / s.rho0 : 0.0);
    m.rho_f = T(1e-12 * s.rho0); m.inv_rho_f = T(1.0 / (1e-12 * s.rho0));
    return m;
}

template <typename T> __host__ __device__ inline T t_exp(T x);
template <> __host__ __device__ inline double t_exp<double>(double x) { return exp(x); }
template <> __host__ __device__ inline float t_exp<float>(float x) { return expf(x); }
template <typename T> __host__ __device__ inline T t_sqrt(T x);
template <> __host__ __device__ inline double t_sqrt<double>(double x) { return sqrt(x); }
template <> __host__ __device__ inline float t_sqrt<float>(float x) { return sqrtf(x); }

// ---------------------------------------------------------------------------------
// Tillotson (1962) equation of state as the paper's SALEc heritage uses it (Sect. 1,
// "various equations of state"): compressed branch, expanded branch with the two
// exponential terms, linear blend in I between E_iv and E_cv.  Returns the pressure
// before the tension cut-off and c^2 = dp/drho + p/rho^2 dp/dI of the branch (in the
// blend, the blend of the two branches' values), floored.
// ---------------------------------------------------------------------------------
// a < b for b > 0 on the bit patterns: an integer compare (any negative a, and -0, is below)
__device__ __forceinline__ bool below_bits(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool below_bits(float a, float b) { return __float_as_int(a) < __float_as_int(b); }
__device__ __forceinline__ bool warp_any(bool p);

template <typename T>
__host__ __device__ __forceinline__ void eos_eval(const MatT<T>& m, T rho_in, T I_in, T& p_out, T& c2_out)
{
    const T zero = T(0), one = T(1), two = T(2);
    const T I = I_in > zero ? I_in : zero;
    if (m.eos == SALEC_EOS_IDEAL_GAS) {
        const T gm1 = m.gamma - one;
        p_out = gm1 * rho_in * I;
        c2_out = m.gamma * gm1 * I;
        return;
    }
    // evaluated at no less than rho_f = 1e-12 rho0, where the form is in its dilute limit:
    // c^2 no longer depends on rho and p is proportional to it (p = a rho I once the
    // exponential terms vanish), so below rho_f the pressure is scaled back by rho / rho_f;
    // the rho^-2 terms below stay finite in FP32
    const T rho = rho_in > m.rho_f ? rho_in : m.rho_f;
    // two divisions: 1/rho and 1/w0 (1/(E0 eta^2) = (rho0^2/E0) / rho^2)
    const T irho = one / rho;
    const T mu = (rho - m.rho0) * m.inv_rho0;
    const T ie = m.rho0sq_E0 * irho * irho;            // 1 / (E0 eta^2)
    const T w0 = I * ie + one;
    const T iw = one / w0;
    const T bw = m.b * iw;                             // b / w0
    const T dw = bw * iw * I * ie;                     // b I / (w0^2 E0 eta^2)
    // compressed branch and its partial derivatives
    const T pc = (m.a + bw) * rho * I + mu * (m.A + m.B * mu);
    const T pc_r = (m.a + bw) * I + two * dw * I + (m.A + two * m.B * mu) * m.inv_rho0;
    const T pc_I = rho * (m.a + bw - dw);
    const T irho2 = irho * irho;
    T p, c2;
    if (rho >= m.rho0 || I <= m.Eiv) {
        p = pc;
        c2 = pc_r + pc * irho2 * pc_I;
    } else {
        const T x = m.rho0 * irho - one;               // rho0/rho - 1
        const T x_r = -m.rho0 * irho * irho;           // dx/drho
        const T ea = t_exp<T>(-m.alpha * x * x);
        const T eb = t_exp<T>(-m.beta * x);
        const T tb = bw * rho * I;                     // b rho I / w0
        const T tb_r = bw * I + two * dw * I;
        const T ta = m.A * mu * eb;
        const T ta_r = m.A * m.inv_rho0 * eb - m.beta * x_r * ta;
        const T tsum = tb + ta;
        const T pe = m.a * rho * I + tsum * ea;
        const T pe_r = m.a * I + (tb_r + ta_r) * ea - two * m.alpha * x * x_r * tsum * ea;
        const T pe_I = m.a * rho + rho * (bw - dw) * ea;
        const T ce2 = pe_r + pe * irho2 * pe_I;
        if (I >= m.Ecv) {
            p = pe;
            c2 = ce2;
        } else {
            // linear blend in I; the sound speed is the same blend of the two branches' own
            // sound speeds (the derivative of the blended pressure would add
            // (p_e - p_c)/(E_cv - E_iv) p/rho^2, unbounded as rho -> 0 when A != B)
            const T we = (I - m.Eiv) * m.inv_dE, wc = (m.Ecv - I) * m.inv_dE;
            p = we * pe + wc * pc;
            c2 = we * ce2 + wc * (pc_r + pc * irho2 * pc_I);
        }
    }
    // a near-empty cell keeps the dilute gas's pressure, not the one at rho_f (whose
    // gradient per unit of so little mass would accelerate it without bound); such cells
    // are rare, so on the GPU the test is an integer compare of the bit patterns (rho_f > 0:
    // a negative rho_in or -0 compares below it too) behind a warp-uniform branch
#ifdef __CUDA_ARCH__
    const bool dilute = below_bits(rho_in, m.rho_f);
    if (warp_any(dilute) && dilute) p *= (rho_in > zero ? rho_in : zero) * m.inv_rho_f;
#else
    if (rho_in < m.rho_f) p *= (rho_in > zero ? rho_in : zero) * m.inv_rho_f;
#endif
    if (!(c2 > m.c2_floor)) c2 = m.c2_floor;
    p_out = p;
    c2_out = c2;
}

template <typename T> __host__ __device__ inline T t_tanh(T x);
template <> __host__ __device__ inline double t_tanh<double>(double x) { return tanh(x); }
template <> __host__ __device__ inline float t_tanh<float>(float x) { return tanhf(x); }

// Rock expanded well below its reference density is fragmented: below rho0 / 2 it carries
// neither shear strength nor tension, between rho0 / 2 and rho0 both are scaled by
// w = 2 rho / rho0 - 1 (in dilute ejecta a stress or tension times a step's strain, per unit
// of so little mass, would send the specific energy to +-1e10 J/kg).
template <typename T>
__host__ __device__ __forceinline__ T expansion_weight(const MatT<T>& m, T rho)
{
    const T w = T(2) * rho * m.inv_rho0 - T(1);
    return w < T(0) ? T(0) : (w > T(1) ? T(1) : w);
}

// Collins et al. (2004) yield strength blended by damage, at max(p, 0), with their thermal
// softening Y tanh(xi (T_m / T - 1)), xi = 1.2, zero at and above melting, and the
// expansion weight.  The state has no temperature: T_m / T is taken as E_iv / I, the
// Tillotson incipient-vaporisation energy standing for the melt energy.  Without it a hot,
// expanded mixture keeps a frictional strength mu p from its vapour pressure and heats
// itself through its stress work.
template <typename T>
__host__ __device__ __forceinline__ T yield_eval(const MatT<T>& m, T p_in, T D, T I, T rho)
{
    const T zero = T(0), one = T(1);
    const T p = p_in > zero ? p_in : zero;
    const T Yi = m.Yi0 + m.mui * p / (one + m.mui * p * m.inv_Yspan);
    T Yd = m.Yd0 + m.mud * p;
    Yd = Yd < m.Ydm ? Yd : m.Ydm;
    T Y = (one - D) * Yi + D * Yd;
    if (I > zero) {
        if (!(I < m.Eiv)) return zero;
        Y *= t_tanh<T>(T(1.2) * (m.Eiv / I - one));
    }
    Y *= expansion_weight(m, rho);
    return Y > zero ? Y : zero;
}

// Sign tests on the bit pattern: integer instructions instead of floating-point compares
// (FP64 compares issue on the FP64 pipe, the bottleneck of the FP64 form).  pos(x): x > 0
// (or +NaN); neg(x): x < 0 (or -NaN), -0 excluded: a resting face (velocity -0)
// moves nothing and costs nothing.
__device__ __forceinline__ bool pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool neg(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool pos(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool neg(float x)
{
    const int b = __float_as_int(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool is_nan(double x)
{
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool is_nan(float x) { return (__float_as_int(x) & 0x7fffffff) > 0x7f800000; }
// x != 0 (either sign of zero counts as zero) on the bit pattern
__device__ __forceinline__ bool nonzero(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ bool is_pzero(double x) { return __double_as_longlong(x) == 0; }
__device__ __forceinline__ bool is_pzero(float x) { return __float_as_int(x) == 0; }
__device__ __forceinline__ bool nonzero(float x) { return (__float_as_int(x) << 1) != 0; }
// Any active lane of the warp: a warp-uniform branch condition.  Guarding FP64 work with it
// keeps the compiler from turning a rarely taken branch into predicated instructions that
// every warp would issue (FP64 instructions occupy the FP64 pipe even when predicated off);
// warps of resting cells then skip them entirely.
__device__ __forceinline__ bool warp_any(bool p) { return __any_sync(__activemask(), p); }
// the step's dt in the element type: the FP32 copy needs no FP64 conversion
template <typename T> __device__ __forceinline__ T step_dt(const DevScalars* s);
template <> __device__ __forceinline__ double step_dt<double>(const DevScalars* s) { return s->dt; }
template <> __device__ __forceinline__ float step_dt<float>(const DevScalars* s) { return s->dtf; }
// max of two non-negative numbers by their bit patterns
__device__ __forceinline__ double max_nonneg(double a, double b)
{
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ float max_nonneg(float a, float b)
{
    return __int_as_float(max(__float_as_int(a), __float_as_int(b)));
}

// launchers (salec_kernels.cu), instantiated for T = double and T = float
template <typename T> cudaError_t launch_step(const ParamsT<T>& P, const dim3* blk, cudaStream_t s, cudaEvent_t* ev);
template <typename T>
cudaError_t launch_batch_step(const ParamsT<T>* runs_dev, int nruns, int nmat, bool strength, bool uniform, const BatchTile* const* work,
                              const int* ntiles, const dim3* blk, cudaStream_t s, cudaEvent_t* ev);
template <typename T> cudaError_t launch_batch_poll(const ParamsT<T>* runs_dev, int n, double* out, cudaStream_t s);
template <typename T>
cudaError_t prepare_batch_persistent(int nmat, bool strength, bool uniform, dim3 blk, int* ctas);
template <typename T>
cudaError_t launch_batch_persistent(const ParamsT<T>* runs, int nruns, int nmat, bool strength, bool uniform,
                                    const BatchTile* cells, int ncells, const BatchTile* verts, int nverts, dim3 blk,
                                    int ctas, int steps, GridSync* gs, bool expire, cudaStream_t s);
template <typename T> cudaError_t launch_courant(const ParamsT<T>& P, cudaStream_t s);
// fused form (salec_fused.cu): after the Courant kernel, the rest-tile kernel and the
// persistent tile kernel.  kFusedTileW x kFusedTileMinH bounds the tile count of every
// instantiation (the rest flags and the work list are sized by it).
constexpr int kFusedTileW = 32, kFusedTileMinH = 16;
template <typename T> cudaError_t prepare_fused(const ParamsT<T>& P, int* ctas);
template <typename T> size_t fused_smem_bytes(const ParamsT<T>& P);
template <typename T> int fused_tiles(const ParamsT<T>& P);
template <typename T> cudaError_t launch_courant_rates(const ParamsT<T>& P, unsigned char* rest, cudaStream_t s);
template <typename T>
cudaError_t launch_step_fused(const ParamsT<T>& P, const OutPtrsT<T>& O, cudaStream_t s, cudaEvent_t* ev);
// The FP64 form's tiles at rest copied beside the tile kernel: a scan kernel queues the
// tiles (as the rest-tile kernel does) and a copy kernel of one warp per SM, on a second
// stream, moves the tiles at rest with bulk tensor copies while the tile kernel runs.  It
// needs a tile-kernel CTA and a copy CTA to fit on one SM together (registers and shared
// memory), even nr (the energy's rows then start on 16-byte boundaries) and a uniform
// grid of one hydrodynamic material.  The maps and the launch shape of one direction
// (read copy -> written copy):
constexpr int kCopyFields = kMaxMat + 2;
struct RestCopy {
    CUtensorMap src[kCopyFields];   // (f, rho) of each material, I, the EoS cache of the copy read
    CUtensorMap dst[kCopyFields];   // the same fields of the copy written
    CUtensorMap v;                  // the vertices of the copy written
    int ctas;                       // one per SM
    int smem;                       // dynamic shared memory of a copy CTA
};
// false (no error pending) where the form is not available for this grid and device
bool prepare_rest_copy(const ParamsT<double>& P, const OutPtrsT<double>& O, RestCopy* rc);
// one step: the Courant kernel on s; then the copy kernel on s2 beside the scan and tile
// kernels on s; s waits for s2 at the end.  With ev: events before the Courant kernel (s),
// after the copy kernel (s2), after the scan kernel (s), after the tile kernel (s).
cudaError_t launch_step_fused_beside(const ParamsT<double>& P, const OutPtrsT<double>& O, const RestCopy& rc,
                                     cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join,
                                     cudaEvent_t* ev);
bool kernel_on_vertices(int k);
int tiles_of(int nr, int nz, int k, dim3 blk);
template <typename T> cudaError_t launch_pressure(const ParamsT<T>& P, double* out, cudaStream_t s);
template <typename T> cudaError_t launch_column_heights(const ParamsT<T>& P, double* heights, cudaStream_t s);
template <typename T> cudaError_t launch_conservation(const ParamsT<T>& P, double* partial4, int* nblocks, cudaStream_t s);
const char* kernel_name(int k);
int launches_per_step();     // timed phases of a step (the Courant kernel is timed within phase 0)
int kernels_per_step();      // kernel launches of a step
const char* noalloc_last_error();
int cell_blocks(int nr, int nz);
int vertex_blocks(int nr, int nz);

}  // namespace salec
