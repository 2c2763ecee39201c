// salec_device.cuh -- device helpers shared by the phase kernels (salec_kernels.cu) and
// the fused tile kernel (salec_fused.cu): block reductions, the absorbing strip's row
// mask, the cell geometry of uniform and non-uniform grids, and the dual-face fluxes of
// the momentum remap.
#pragma once

#include "salec_internal.cuh"

namespace salec {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum, result valid in thread 0 (blocks are whole warps, at most kMaxThreads)
static __device__ double block_sum(double v, double* sh)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < nw; ++w) s += sh[w];
    return s;
}

// The right absorbing strip acts on the rows whose reference (far-field) state holds
// material: the medium whose waves it absorbs.  Above the target the reference is void and
// damping toward it would remove ejecta, so there it does nothing (cells: row j; vertices:
// either adjacent cell row).
template <typename T>
__device__ __forceinline__ bool strip_row_c(const PtrsT<T>& p, int j) { return pos(p.rho_ref[j]); }
template <typename T>
__device__ __forceinline__ bool strip_row_v(const PtrsT<T>& p, int j, int nz)
{
    return (j > 0 && pos(p.rho_ref[j - 1])) || (j < nz && pos(p.rho_ref[j]));
}

// ---------------------------------------------------------------------------------
// Cell geometry per radian.  A non-uniform grid (UNI = false) takes a cell's volume and
// radial faces as a column entry times its row height: V = r_c dr dz, A_R = r_i dz; a
// uniform grid of dx cells (UNI = true) keeps one entry per column for every row, which
// spares the FP64 pipe those products.
// ---------------------------------------------------------------------------------
template <typename T, bool UNI>
struct Geo {
    static __device__ __forceinline__ T vol(const ParamsT<T>& P, int i, int j)
    {
        return UNI ? P.p.V[i] : P.p.A_Z[i] * P.p.dz[j];
    }
    static __device__ __forceinline__ T ivol(const ParamsT<T>& P, int i, int j)
    {
        return UNI ? P.p.invV[i] : P.p.invAZ[i] * P.p.idz[j];
    }
    // radial face area at r_i of row j
    static __device__ __forceinline__ T area_r(const ParamsT<T>& P, int i, int j)
    {
        return UNI ? P.p.A_R[i] : P.p.rR[i] * P.p.dz[j];
    }
    // net radial volume flux A_R(i+1) uR - A_R(i) uL of cell (i,j)
    static __device__ __forceinline__ T flux_r(const ParamsT<T>& P, int i, int j, T uL, T uR)
    {
        return UNI ? P.p.A_R[i + 1] * uR - P.p.A_R[i] * uL : P.p.dz[j] * (P.p.rR[i + 1] * uR - P.p.rR[i] * uL);
    }
    static __device__ __forceinline__ T idr(const ParamsT<T>& P, int i) { return UNI ? P.idx : P.p.idr[i]; }
    static __device__ __forceinline__ T idz(const ParamsT<T>& P, int j) { return UNI ? P.idx : P.p.idz[j]; }
    // the cell's length scale L = min(dr, dz) and 1 / L
    static __device__ __forceinline__ T len(const ParamsT<T>& P, int i, int j)
    {
        if (UNI) return P.dx;
        const T a = P.p.dr[i], b = P.p.dz[j];
        return a < b ? a : b;
    }
    static __device__ __forceinline__ T ilen(const ParamsT<T>& P, int i, int j)
    {
        if (UNI) return P.idx;
        const T a = P.p.idr[i], b = P.p.idz[j];
        return a > b ? a : b;
    }
    // derivatives of the cell's stress power V S:e with respect to its corner velocities:
    // V / (2 dr) for r-derivatives, V / (4 r_c) for the hoop strain rate
    static __device__ __forceinline__ T half_v_dr(const ParamsT<T>& P, int i, int j)
    {
        return UNI ? T(0.5) * P.p.A_Z[i] : T(0.5) * P.p.rc[i] * P.p.dz[j];
    }
    static __device__ __forceinline__ T quarter_v_rc(const ParamsT<T>& P, int i, int j)
    {
        return UNI ? T(0.25) * P.dx2 : T(0.25) * P.p.dr[i] * P.p.dz[j];
    }
};

// What a dual face carries: mass f, momentum f w and kinetic energy f |w|^2 / 2 with the
// upwind vertex velocity w.
template <typename T>
struct DualFace {
    T f, fr, fz, e;
};
// products rounded as written (never fused into a multiply-add with their later use), so
// that a face computed by either of its vertices, or read from the other, is the same
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
template <typename T>
__device__ __forceinline__ DualFace<T> dual_face(T f, typename VT<T>::T2 w)
{
    DualFace<T> d;
    d.f = f;
    d.fr = mul_rn(f, w.x);
    d.fz = mul_rn(f, w.y);
    d.e = mul_rn(mul_rn(T(0.5), f), add_rn(mul_rn(w.x, w.x), mul_rn(w.y, w.y)));
    return d;
}

// Net fluxes of a cell's remap: material volumes and masses, stress and damage contents,
// and the energy change of the inflows.
template <typename T, int NM>
struct Acc {
    T Vm[NM], Mm[NM], S[4];
    T dI;        // sum over inflows of (I_donor - I^L) * mass (the remap's energy change)
};

}  // namespace salec
