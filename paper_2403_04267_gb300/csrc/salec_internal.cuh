// salec_internal.cuh -- shared definitions of the CUDA library: parameter blocks passed
// to the kernels by value, the device-state layout, and the material laws used on both
// the host (set-up) and the device (time step).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/salec.h"

namespace salec {

constexpr int kMaxMat = 3;
constexpr int kBlockX = 32;
constexpr int kBlockY = 8;
constexpr int kThreads = kBlockX * kBlockY;

// Material constants with the derived quantities the kernels use.
struct Mat {
    int eos, strength;
    double rho0, inv_rho0, rho0sq_E0, A, B, E0, a, b, alpha, beta, Eiv, Ecv, inv_dE, gamma;
    double Yi0, mui, Yim, Yd0, mud, Ydm, inv_Yspan, G, eps_fb, B_dam, p_bd, p_t, c2_floor;
};

// Scalars of a run, resident on the device.
struct DevScalars {
    double t, dt, dt_prev, pad0;
    double mass_out, mass_discarded, mass_pml, zmom_out;
    unsigned long long nstep;
    unsigned int counter;   // last-block counter of the dt reduction
    int status;             // bit 1: non-positive volume or density, 2: NaN, 4: dt < dt_min
};

// Device pointers into the caller's state buffer.
struct Ptrs {
    // persistent cell state
    double2* fr[kMaxMat];   // (f_m, rho_m)
    double* I;              // specific internal energy
    double2* s01;           // (s_rr, s_zz)        [strength only]
    double2* s2d;           // (s_rz, D)           [strength only]
    double* pmax;           // running peak over-pressure
    double2* v;             // vertex (v_r, v_z)
    // PML auxiliaries (compact strips)
    double2* pb_c;          // bottom cells (phi1, phi3), index j*nr + i, j < pb
    double* pb_psi2;        // bottom cells psi2
    double4_32a* pb_v;      // bottom vertices (phi2r, phi2z, psi1r, psi1z), index j*(nr+1)+i, j < pb
    double2* pr_c;          // right cells (phi1, phi3), index j*pr + (i - (nr - pr))
    double* pr_psi2;
    double4_32a* pr_v;      // right vertices, index j*pr + (i - (nr - pr + 1)), i > nr - pr
    // tables
    const double* A_R;      // nr+1 radial face areas
    const double* A_Z;      // nr vertical face areas
    const double* V;        // nr cell volumes
    const double* invV;     // nr
    const double* inv2rc;   // nr  1 / (2 r_c)
    const double* p0;       // nz reference pressure per row
    const double* rho_ref;  // nz
    const double* I_ref;    // nz
    const double* dB_c;     // nz   bottom-strip profile at cell centres
    const double* dB_v;     // nz+1 bottom-strip profile at vertices
    const double* dR_c;     // nr
    const double* dR_v;     // nr+1
    // per-step scratch
    double2* PM;            // (P, M) per cell
    double2* pbphi;         // (p_bar, Phi) per cell
    double2* vL;            // Lagrangian vertex velocity
    double* mv;             // vertex mass
    double* dK;             // Lagrangian kinetic-energy deficit per vertex
    double* kheat;          // specific heat returned per vertex
    double2* frL[kMaxMat];  // Lagrangian (f_m^L, rho_m^L)
    double2* VIL;           // (V^L, I^L)
    double2* sL01;          // Lagrangian (s_rr, s_zz)
    double2* sL2d;          // Lagrangian (s_rz, D)
    double* dMR;            // signed mass flux through radial faces, (nr+1) x nz
    double* dMZ;            // signed mass flux through vertical faces, nr x (nz+1)
    double* partial;        // per-block reduction partials
    DevScalars* scal;
};

struct Params {
    int nr, nz, nmat, pr, pb, bc_top, bc_bottom, any_strength, nblk_cells;
    double dx, dx2, cfl, growth, dt_max, dt_min, g, cq, cl, f_min;
    Mat mat[kMaxMat];
    Ptrs p;
};

// ---------------------------------------------------------------------------------
// Tillotson (1962) equation of state as the paper's SALEc heritage uses it (Sect. 1,
// "various equations of state"): compressed branch, expanded branch with the two
// exponential terms, linear blend in I between E_iv and E_cv.  Returns the pressure
// before the tension cut-off and c^2 = dp/drho + p/rho^2 dp/dI (floored).
// ---------------------------------------------------------------------------------
__host__ __device__ inline void eos_eval(const Mat& m, double rho, double I_in, double& p_out, double& c2_out)
{
    const double I = I_in > 0.0 ? I_in : 0.0;
    if (m.eos == SALEC_EOS_IDEAL_GAS) {
        const double gm1 = m.gamma - 1.0;
        p_out = gm1 * rho * I;
        c2_out = m.gamma * gm1 * I;
        return;
    }
    // two divisions: 1/rho and 1/w0 (1/(E0 eta^2) = (rho0^2/E0) / rho^2)
    const double irho = 1.0 / rho;
    const double mu = (rho - m.rho0) * m.inv_rho0;
    const double ie = m.rho0sq_E0 * irho * irho;        // 1 / (E0 eta^2)
    const double w0 = I * ie + 1.0;
    const double iw = 1.0 / w0;
    const double bw = m.b * iw;                         // b / w0
    const double dw = bw * iw * I * ie;                 // b I / (w0^2 E0 eta^2)
    // compressed branch and its partial derivatives
    const double pc = (m.a + bw) * rho * I + mu * (m.A + m.B * mu);
    const double pc_r = (m.a + bw) * I + 2.0 * dw * I + (m.A + 2.0 * m.B * mu) * m.inv_rho0;
    const double pc_I = rho * (m.a + bw - dw);
    double p, p_r, p_I;
    if (rho >= m.rho0 || I <= m.Eiv) {
        p = pc; p_r = pc_r; p_I = pc_I;
    } else {
        const double x = m.rho0 * irho - 1.0;            // rho0/rho - 1
        const double x_r = -m.rho0 * irho * irho;        // dx/drho
        const double ea = exp(-m.alpha * x * x);
        const double eb = exp(-m.beta * x);
        const double tb = bw * rho * I;                  // b rho I / w0
        const double tb_r = bw * I + 2.0 * dw * I;
        const double ta = m.A * mu * eb;
        const double ta_r = m.A * m.inv_rho0 * eb - m.beta * x_r * ta;
        const double tsum = tb + ta;
        const double pe = m.a * rho * I + tsum * ea;
        const double pe_r = m.a * I + (tb_r + ta_r) * ea - 2.0 * m.alpha * x * x_r * tsum * ea;
        const double pe_I = m.a * rho + rho * (bw - dw) * ea;
        if (I >= m.Ecv) {
            p = pe; p_r = pe_r; p_I = pe_I;
        } else {
            const double we = (I - m.Eiv) * m.inv_dE, wc = (m.Ecv - I) * m.inv_dE;
            p = we * pe + wc * pc;
            p_r = we * pe_r + wc * pc_r;
            p_I = we * pe_I + wc * pc_I + (pe - pc) * m.inv_dE;
        }
    }
    double c2 = p_r + p * irho * irho * p_I;
    if (!(c2 > m.c2_floor)) c2 = m.c2_floor;
    p_out = p;
    c2_out = c2;
}

// Collins et al. (2004) yield strength blended by damage, at max(p, 0).
__host__ __device__ inline double yield_eval(const Mat& m, double p_in, double D)
{
    const double p = p_in > 0.0 ? p_in : 0.0;
    const double Yi = m.Yi0 + m.mui * p / (1.0 + m.mui * p * m.inv_Yspan);
    double Yd = m.Yd0 + m.mud * p;
    Yd = Yd < m.Ydm ? Yd : m.Ydm;
    const double Y = (1.0 - D) * Yi + D * Yd;
    return Y > 0.0 ? Y : 0.0;
}

// launchers (salec_kernels.cu)
cudaError_t launch_step(const Params& P, cudaStream_t s, cudaEvent_t* ev);
const char* kernel_name(int k);
cudaError_t launch_pressure(const Params& P, double* out, cudaStream_t s);
cudaError_t launch_column_heights(const Params& P, double* heights, cudaStream_t s);
cudaError_t launch_conservation(const Params& P, double* partial4, int* nblocks, cudaStream_t s);
int launches_per_step();
const char* noalloc_last_error();
int cell_blocks(int nr, int nz);
int vertex_blocks(int nr, int nz);

}  // namespace salec

namespace salec {
// Sign tests on the bit pattern: integer instructions instead of FP64 compares (which
// issue on the FP64 pipe, the bottleneck of the FP64 form).  pos(x): x > 0 (or +NaN);
// neg(x): x < 0 or x == -0.0 (callers treat -0.0 like 0 by moving zero volume).
__device__ __forceinline__ bool pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool neg(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool is_nan(double x)
{
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}
// max of two non-negative doubles by their bit patterns
__device__ __forceinline__ double max_nonneg(double a, double b)
{
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
}  // namespace salec
