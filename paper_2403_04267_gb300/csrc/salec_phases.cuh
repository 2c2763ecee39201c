// salec_phases.cuh -- the bodies of the six phases of the SALE cycle on sm_103a, for the
// FP64 form (T = double) and the mixed form (T = float, FP64 specific internal energy).
// Each body computes one block of cells or vertices given the block's coordinates, so the
// single-run kernels, the batched kernels (salec_kernels.cu) and the persistent batched
// kernel (salec_persist.cu) run the same code per cell and vertex.
//
//   phase 0   EoS, tension cut-off, artificial viscosity, Courant reduction (block max of
//             |v| + c into a per-run atomic maximum)                     Eqs. 1-2, Eq. 14
//   phase 1   vertex corner forces incl. hoop stress, gravity, PML psi1, v^L, BCs  Eq. 1, Eqs. 16/21
//   phase 2   swept volumes, strain rates, compatible energy, PML psi2, void/material
//             volume partition, Jaumann + von Mises + damage        Eq. 2, Eqs. 17/22
//   phase 3a  donor-cell VOF remap, clean-up, PML phi1/phi3 + damping   Eqs. 3, 5, 18, 20, 23, 25
//   phase 3b  dual-grid momentum remap, PML phi2 + damping, KE deficit  Eqs. 4, 19, 24
//   phase 3c  kinetic-energy deficit returned as heat; time advance
//
// Layout: cell arrays row-major [j][i] (nr fastest), vertex arrays [j][i] over nr+1;
// paired quantities are 2-vectors so one warp moves contiguous 256 or 512 bytes per load.
// In templated code every literal is T(...) so the FP32 form issues no FP64 arithmetic
// except in the energy update and the reductions.
//
// Barriers: every barrier of a body is reached by every thread of the block (a thread
// outside the grid leaves a body only where no barrier follows), so one block may run
// several bodies in a row with a barrier between them.
#pragma once
#include <cuda_runtime.h>

#include "salec_device.cuh"

namespace salec {

// ---------------------------------------------------------------------------------
// Phase 0: equation of state, artificial viscosity and the Courant time step.
// ---------------------------------------------------------------------------------
template <typename T, int NM, bool STR, bool UNI>
__device__ __forceinline__ void body_phase0(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    typedef Geo<T, UNI> GE;
    const T zero = T(0), one = T(1), half = T(0.5);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr;
    const PtrsT<T>& p = P.p;
    // largest (|v| + c) / L of the block, L = min(dr, dz) the cell's length scale: the
    // min over cells of L / (|v| + c) is C0 over its max, one division per step (a
    // uniform grid takes the max of |v| + c and divides dx by it).  The max is exact in T,
    // so it is taken in T and the block's value converted to FP64 once.
    T speed = zero;
    if (i < nr && j < P.nz) {
        const int c = j * nr + i;
        T phat = zero, phi = zero, mass = zero, c2m = zero, p1 = zero, r1 = zero;
        const T Ic = T(p.I[c]);
        const T D = STR ? p.s2d[c].y : zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const typename V::T2 fr = p.fr[m][c];
            if (pos(fr.x)) {
                T pm, c2;
                eos_eval<T>(P.mat[m], fr.y, Ic, pm, c2);
                const T pmin = (one - D) * P.mat[m].p_t * expansion_weight(P.mat[m], fr.y);
                pm = pm < pmin ? pmin : pm;
                phat += fr.x * pm;
                phi += fr.x;
                mass += fr.x * fr.y;
                c2m = max_nonneg(c2m, c2);
                p1 = pm;
                r1 = fr.y;
            }
        }
        T Pc = zero, pbar = zero;
        if (pos(phi)) {
            const int nv = nr + 1;
            const typename V::T2 va = p.v[j * nv + i], vb = p.v[j * nv + i + 1];
            const typename V::T2 vc = p.v[(j + 1) * nv + i + 1], vd = p.v[(j + 1) * nv + i];
            const T uL = half * (va.x + vd.x), uR = half * (vb.x + vc.x);
            const T uB = half * (va.y + vb.y), uT = half * (vd.y + vc.y);
            const T div = (GE::flux_r(P, i, j, uL, uR) + p.A_Z[i] * (uT - uB)) * GE::ivol(P, i, j);
            const T cs = t_sqrt<T>(c2m);
            // one material: p_bar = p and rho_bar = rho; otherwise divide by Phi once
            const T iphi = NM == 1 ? one : one / phi;
            pbar = NM == 1 ? p1 : phat * iphi;
            T q = zero;
            if (neg(div)) {
                const T rb = NM == 1 ? r1 : mass * iphi;
                const T L = GE::len(P, i, j);
                q = rb * (P.cq * (UNI ? P.dx2 : L * L) * div * div - P.cl * L * cs * div);
            }
            Pc = phat + phi * q;
            const T over = pbar - p.p0[j];
            if (over > p.pmax[c]) p.pmax[c] = over;
            T w = va.x * va.x + va.y * va.y;
            w = max_nonneg(w, vb.x * vb.x + vb.y * vb.y);
            w = max_nonneg(w, vc.x * vc.x + vc.y * vc.y);
            w = max_nonneg(w, vd.x * vd.x + vd.y * vd.y);
            speed = t_sqrt<T>(w) + cs;
            if (!UNI) speed = speed * GE::ilen(P, i, j);
            if (is_nan(speed)) atomicOr(&p.scal->status, 2);
        }
        p.PM[c] = V::mk(Pc, mass * GE::vol(P, i, j));
        p.pbphi[c] = V::mk(pbar, phi);
    }
    // block maximum (on the bit patterns of the non-negative speeds) into one running
    // maximum per run by an atomic max that nothing waits for; the Courant kernel that
    // follows turns it into dt.  After the one barrier only thread 0 works, so the other
    // warps leave at once and the block right after its atomic.
    __shared__ unsigned long long sh[kMaxThreads / 32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    for (int o = 16; o > 0; o >>= 1) speed = max_nonneg(speed, __shfl_down_sync(0xffffffffu, speed, o));
    if ((tid & 31) == 0) sh[tid >> 5] = (unsigned long long)__double_as_longlong(double(speed));
    __syncthreads();
    if (tid != 0) return;
    unsigned long long b = sh[0];
    for (int w = 1; w < nw; ++w) b = max(b, sh[w]);
    atomicMax(&p.scal->maxbits, b);
}

// Courant step of Eq. 14 from phase 0's running maximum of (|v| + c) / L (of |v| + c on a
// uniform grid): dt = min(C0 / max, growth dt_prev, dt_max); the maximum is reset for the
// next step.  One thread per run.
template <typename T>
__device__ __forceinline__ void courant_dt(const ParamsT<T>& P)
{
    DevScalars* s = P.p.scal;
    const double mx = __longlong_as_double((long long)s->maxbits);
    s->maxbits = 0ull;
    double dt = P.growth * s->dt_prev;
    const double cdt = P.uniform ? P.cfld * (P.dxd / mx) : P.cfld / mx;
    dt = cdt < dt ? cdt : dt;
    dt = P.dt_max < dt ? P.dt_max : dt;
    if (dt < P.dt_min) s->status |= 4;
    s->dt = dt;
    s->dtf = float(dt);
    s->active = 1;
}

// ---------------------------------------------------------------------------------
// Phase 1: corner forces, gravity and PML psi1 on the vertices; Lagrangian velocity.
// Cells around vertex (i,j): k = 0 (i-1,j-1) corner c, 1 (i,j-1) corner d,
// 2 (i,j) corner a, 3 (i-1,j) corner b.
// ---------------------------------------------------------------------------------
template <typename T, bool STR, bool UNI>
__device__ __forceinline__ void body_phase1(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    typedef Geo<T, UNI> GE;
    const T zero = T(0), one = T(1), half = T(0.5);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    if (i > nr || j > nz) return;
    const PtrsT<T>& p = P.p;
    const T dt = step_dt<T>(p.scal);
    const int v = j * (nr + 1) + i;
    T Pc[4] = {zero, zero, zero, zero}, Pp[4] = {zero, zero, zero, zero};
    T devr_rad = zero, devz_rad = zero, devr_ver = zero, devz_ver = zero, mass = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ci = (k == 0 || k == 3) ? i - 1 : i;
        const int cj = (k < 2) ? j - 1 : j;
        if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
        const int c = cj * nr + ci;
        const typename V::T2 pm = p.PM[c];
        Pc[k] = pm.x;
        mass += T(0.25) * pm.y;
        if (STR || P.pr > 0 || P.pb > 0) {
            const T phi = p.pbphi[c].y;
            Pp[k] = pm.x - phi * p.p0[cj];
            if (STR) {
                const typename V::T2 s01 = p.s01[c];
                const T srz = p.s2d[c].x;
                const T Srr = phi * s01.x, Szz = phi * s01.y, Srz = phi * srz;
                const T Stt = -(Srr + Szz);
                // corner-velocity derivatives of the stress power: V / (2 dr), V / (2 dz)
                // for r- and z-derivatives, V / (4 r_c) for the hoop strain rate
                const T hr = GE::half_v_dr(P, ci, cj), hz = half * p.A_Z[ci];
                const T hoop = GE::quarter_v_rc(P, ci, cj);
                // a (k=2), d (k=1) on the left face; a, b (k=3) at the bottom of the cell
                const T sr = (k == 2 || k == 1) ? one : -one;
                const T sz = (k == 2 || k == 3) ? one : -one;
                devr_rad += sr * hr * Srr - hoop * Stt;
                devz_rad += sr * hr * Srz;
                devr_ver += sz * hz * Srz;
                devz_ver += sz * hz * Szz;
            }
        }
    }
    // radial faces at r_i of rows j-1 (cells 0, 1) and j (cells 3, 2); one area when every
    // row has the same height
    const T ARb = UNI ? p.A_R[i] : (j > 0 ? GE::area_r(P, i, j - 1) : zero);
    const T ARt = UNI ? ARb : (j < nz ? GE::area_r(P, i, j) : zero);
    const T AZl = i > 0 ? p.A_Z[i - 1] : zero, AZr = i < nr ? p.A_Z[i] : zero;
    const T Fr = (UNI ? half * ARb * (((Pc[0] + Pc[3]) - Pc[1]) - Pc[2])
                      : half * (ARb * (Pc[0] - Pc[1]) + ARt * (Pc[3] - Pc[2]))) + (devr_rad + devr_ver);
    const T Fz = half * (AZl * (Pc[0] - Pc[3]) + AZr * (Pc[1] - Pc[2])) + (devz_rad + devz_ver);
    T psr = zero, psz = zero;
    if (j < P.pb) {
        const T d = p.dB_v[j];
        typename V::T4 a = p.pb_v[v];
        const T Tr = (UNI ? half * ARb * (((Pp[0] + Pp[3]) - Pp[1]) - Pp[2])
                          : half * (ARb * (Pp[0] - Pp[1]) + ARt * (Pp[3] - Pp[2]))) + devr_rad;
        const T rl = one - P.alpha_b * dt;     // relaxation of the auxiliaries
        a.z = a.z * rl - dt * d * Tr;
        a.w = a.w * rl - dt * d * devz_rad;
        p.pb_v[v] = a;
        psr += a.z; psz += a.w;
    }
    if (i > nr - P.pr) {
        const int k = j * P.pr + (i - (nr - P.pr + 1));
        const T d = strip_row_v(p, j, P.nz) ? p.dR_v[i] : zero;
        typename V::T4 a = p.pr_v[k];
        const T Tz = half * (AZl * (Pp[0] - Pp[3]) + AZr * (Pp[1] - Pp[2])) + devz_ver;
        const T rl = one - P.alpha_r * dt;
        a.z = a.z * rl - dt * d * devr_ver;
        a.w = a.w * rl - dt * d * Tz;
        p.pr_v[k] = a;
        psr += a.z; psz += a.w;
    }
    const typename V::T2 vn = p.v[v];
    T vr = zero, vz = zero;
    if (pos(mass)) {
        // no net force and no gravity: v^L = v (the update's own value, up to the sign of a
        // zero) without the reciprocal, which is a long FP64-pipe sequence in the FP64 form
        const T fr_ = Fr - psr, fz_ = Fz - psz;
        const bool acc = nonzero(fr_) || nonzero(fz_) || nonzero(P.g);
        if (warp_any(acc) && acc) {
            const T im = one / mass;
            vr = vn.x + dt * (fr_ * im);
            vz = vn.y + dt * (fz_ * im - P.g);
        } else {
            vr = vn.x;
            vz = vn.y;
        }
    }
    if (i == 0 || i == nr) vr = zero;
    if (j == 0) {
        vz = zero;
        if (P.bc_bottom == SALEC_BOTTOM_NOSLIP) vr = zero;
    }
    if (j == nz && P.bc_top == SALEC_TOP_WALL) vz = zero;
    p.vL[v] = V::mk(vr, vz);
    p.mv[v] = mass;
    const T dvr = vr - vn.x, dvz = vz - vn.y;
    p.dK[v] = half * mass * (dvr * dvr + dvz * dvz);
}

// ---------------------------------------------------------------------------------
// Phase 2: Lagrangian cell update from v^L.
// ---------------------------------------------------------------------------------
template <typename T, int NM, bool STR, bool UNI>
__device__ __forceinline__ void body_phase2(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    typedef Geo<T, UNI> GE;
    const T zero = T(0), one = T(1), half = T(0.5), two = T(2);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr;
    if (i >= nr || j >= P.nz) return;
    const PtrsT<T>& p = P.p;
    const int c = j * nr + i;
    const T phi = p.pbphi[c].y;
    if (!pos(phi)) {
#pragma unroll
        for (int m = 0; m < NM; ++m) p.frL[m][c] = V::mk(zero, zero);
        p.VL[c] = GE::vol(P, i, j);
        p.IL[c] = 0.0;
        if (STR) { p.sL01[c] = V::mk(zero, zero); p.sL2d[c] = V::mk(zero, zero); }
        return;
    }
    const T dt = step_dt<T>(p.scal);
    const int nv = nr + 1;
    const typename V::T2 va = p.vL[j * nv + i], vb = p.vL[j * nv + i + 1];
    const typename V::T2 vc = p.vL[(j + 1) * nv + i + 1], vd = p.vL[(j + 1) * nv + i];
    const T uL = half * (va.x + vd.x), uR = half * (vb.x + vc.x);
    const T uB = half * (va.y + vb.y), uT = half * (vd.y + vc.y);
    const T idr = GE::idr(P, i), idz = GE::idz(P, j);
    const T err = (uR - uL) * idr;
    const T ezz = (uT - uB) * idz;
    const T Vc = GE::vol(P, i, j);
    const T ett = (uR + uL) * p.inv2rc[i];
    const T rad_flux = GE::flux_r(P, i, j, uL, uR);
    const T ver_flux = p.A_Z[i] * (uT - uB);
    const T dV = dt * (rad_flux + ver_flux);
    const T VLc = Vc + dV;
    const typename V::T2 pm = p.PM[c];
    const T Pc = pm.x, M = pm.y;
    T work = zero, Pi_rad = -Pc * rad_flux, Pi_ver = -Pc * ver_flux;
    T dvr_dz = zero, dvz_dr = zero, srr = zero, szz = zero, srz = zero, D = zero;
    if (STR) {
        const typename V::T2 s01 = p.s01[c], s2d = p.s2d[c];
        srr = s01.x; szz = s01.y; srz = s2d.x; D = s2d.y;
        dvr_dz = half * ((vd.x + vc.x) - (va.x + vb.x)) * idz;
        dvz_dr = half * ((vb.y + vc.y) - (va.y + vd.y)) * idr;
        const T Srr = phi * srr, Szz = phi * szz, Srz = phi * srz, Stt = -(Srr + Szz);
        const T erz = half * (dvr_dz + dvz_dr);
        work = dt * Vc * (Srr * err + Szz * ezz + Stt * ett + two * Srz * erz);
        Pi_rad += Vc * (Srr * err + Stt * ett + Srz * dvz_dr);
        Pi_ver += Vc * (Szz * ezz + Srz * dvr_dz);
    }
    T psi2 = zero;
    if (j < P.pb) {
        T a = p.pb_psi2[c];
        a = a * (one - P.alpha_b * dt) - dt * p.dB_c[j] * Pi_rad;
        p.pb_psi2[c] = a;
        psi2 += a;
    }
    if (i >= nr - P.pr) {
        const int k = j * P.pr + (i - (nr - P.pr));
        T a = p.pr_psi2[k];
        a = a * (one - P.alpha_r * dt) - dt * (strip_row_c(p, j) ? p.dR_c[i] : zero) * Pi_ver;
        p.pr_psi2[k] = a;
        psi2 += a;
    }
    const T dE = -Pc * dV + work - dt * psi2;
    const double Ic = p.I[c];
    // the specific internal energy is accumulated in FP64 in every form
    // no energy change: no FP64 instruction (the sum would return Ic unchanged)
    const bool add_dE = pos(M) && nonzero(dE);
    double ILnew = Ic;
    if (warp_any(add_dE) && add_dE) ILnew = Ic + double(dE / M);
    p.IL[c] = ILnew;
    p.VL[c] = VLc;
    // volume partition: matter and void share every volume change in proportion to their
    // fractions (equal strain), so each material's work -p_m dV_m adds up to the -P dV the
    // energy update charges
    const T dVmat = phi * dV;
    bool bad = false;
    T G = zero, Y = zero, iepsf = zero;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const typename V::T2 fr = p.fr[m][c];
        if (pos(fr.x)) {
            const T Vm = fr.x * Vc;
            // one material: f_m / Phi = 1; true divisions keep a resting cell exact
            const T VmL = NM == 1 ? Vm + dVmat : Vm + fr.x / phi * dVmat;
            bad |= !pos(VmL) || !pos(fr.y);     // non-positive Lagrangian volume or density
            // unchanged volume: V_m / V_m^L is exactly 1 (no division)
            p.frL[m][c] = V::mk(VmL / VLc, warp_any(nonzero(dV)) ? fr.y * (Vm / VmL) : fr.y);
            if (STR && P.mat[m].strength == SALEC_STRENGTH_COLLINS) {
                const MatT<T>& mm = P.mat[m];
                const T pb = p.pbphi[c].x;
                G += fr.x * mm.G;
                Y += fr.x * yield_eval<T>(mm, pb, D, T(Ic), fr.y);
                T ef = mm.B_dam * (pb - mm.p_bd);
                ef = ef < mm.eps_fb ? mm.eps_fb : ef;
                iepsf += fr.x / ef;
            }
        } else {
            p.frL[m][c] = V::mk(zero, zero);
        }
    }
    if (bad) atomicOr(&p.scal->status, 1);
    if (STR) {
        const T iphi = one / phi;
        G *= iphi; Y *= iphi; iepsf *= iphi;
        if (pos(G)) {
            const T omega = half * (dvr_dz - dvz_dr);
            const T erz = half * (dvr_dz + dvz_dr);
            const T tr3 = (err + ezz + ett) * (one / T(3));
            const T G2 = two * G;
            T nrr = srr + dt * (G2 * (err - tr3) + two * omega * srz);
            T nzz = szz + dt * (G2 * (ezz - tr3) - two * omega * srz);
            T nrz = srz + dt * (G2 * erz + omega * (szz - srr));
            const T ntt = -(nrr + nzz);
            const T J2 = half * (nrr * nrr + nzz * nzz + ntt * ntt) + nrz * nrz;
            if (J2 > Y * Y) {
                const T sq = t_sqrt<T>(J2);
                const T k = Y / sq;
                nrr *= k; nzz *= k; nrz *= k;
                D += (sq - Y) / (T(1.7320508075688772) * G) * iepsf;
                D = D > one ? one : D;
            }
            srr = nrr; szz = nzz; srz = nrz;
        } else {
            srr = zero; szz = zero; srz = zero;
        }
        p.sL01[c] = V::mk(srr, szz);
        p.sL2d[c] = V::mk(srz, D);
    }
}

// ---------------------------------------------------------------------------------
// Phase 3a: donor-cell remap of the cells.
// ---------------------------------------------------------------------------------

// Swept volume of the radial face at r_i of row j, and of the vertical face at z_j of
// column i, from the Lagrangian velocities (computed identically by both neighbours).
template <typename T, bool UNI>
__device__ __forceinline__ T radial_dV(const ParamsT<T>& P, int i, int j, T dt)
{
    if (i == 0 || i == P.nr) return T(0);
    const int nv = P.nr + 1;
    const T u = T(0.5) * (P.p.vL[j * nv + i].x + P.p.vL[(j + 1) * nv + i].x);
    return dt * Geo<T, UNI>::area_r(P, i, j) * u;
}
template <typename T>
__device__ __forceinline__ T vertical_dV(const ParamsT<T>& P, int i, int j, T dt)
{
    if (j == 0) return T(0);
    if (j == P.nz && P.bc_top == SALEC_TOP_WALL) return T(0);
    const int nv = P.nr + 1;
    const T u = T(0.5) * (P.p.vL[j * nv + i].y + P.p.vL[j * nv + i + 1].y);
    return dt * P.p.A_Z[i] * u;
}

// Flux of |dV| of the donor cell's Lagrangian contents, added with sign sgn to acc.
// Returns the moved mass and energy (energy for the PML auxiliaries only); an inflow
// (sgn > 0) adds (I_donor - I_self) * mass to the energy change.
template <typename T, int NM, bool STR>
__device__ __forceinline__ void move(const ParamsT<T>& P, int donor, T adV, T sgn, double Iself, bool strip,
                                     Acc<T, NM>& acc, T& mass_out, T& e_out)
{
    typedef VT<T> V;
    const PtrsT<T>& p = P.p;
    T vmat = T(0), mass = T(0);
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const typename V::T2 fl = p.frL[m][donor];
        const T dv = adV * fl.x;
        const T dm = fl.y * dv;
        acc.Vm[m] += sgn * dv;
        acc.Mm[m] += sgn * dm;
        vmat += dv;
        mass += dm;
    }
    const double Id = p.IL[donor];
    if (pos(sgn)) acc.dI += T(Id - Iself) * mass;
    if (STR) {
        const typename V::T2 a = p.sL01[donor], b = p.sL2d[donor];
        acc.S[0] += sgn * (a.x * vmat);
        acc.S[1] += sgn * (a.y * vmat);
        acc.S[2] += sgn * (b.x * vmat);
        acc.S[3] += sgn * (b.y * vmat);
    }
    mass_out = mass;
    e_out = strip ? T(Id) * mass : T(0);
}

template <typename T, int NM, bool STR, bool UNI>
__device__ __forceinline__ void body_phase3a(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    const T zero = T(0), one = T(1);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    const PtrsT<T>& p = P.p;
    double t_out = 0.0, t_disc = 0.0, t_pml = 0.0;
    if (i < nr && j < nz) {
        const int c = j * nr + i;
        const T dt = step_dt<T>(p.scal);
        // acc collects the net fluxes; the Lagrangian contents are added back below
        Acc<T, NM> acc;
        const T VLc = p.VL[c];
        const double ILc = p.IL[c];
#pragma unroll
        for (int m = 0; m < NM; ++m) { acc.Vm[m] = zero; acc.Mm[m] = zero; }
        acc.dI = zero;
        acc.S[0] = acc.S[1] = acc.S[2] = acc.S[3] = zero;
        // net tangential outflows for the PML auxiliaries: radial (bottom strip), vertical (right strip)
        const bool strip = j < P.pb || i >= nr - P.pr;
        T FRm = zero, FRe = zero, FZm = zero, FZe = zero;
        T fm, fe;
        // left face r_i: positive dV flows from (i-1,j) into this cell
        {
            const T dV = radial_dV<T, UNI>(P, i, j, dt);
            T sm = zero;
            if (!warp_any(nonzero(dV))) {
            } else if (pos(dV)) { move<T, NM, STR>(P, c - 1, dV, one, ILc, strip, acc, fm, fe); sm = fm; FRm -= fm; FRe -= fe; }
            else if (neg(dV)) { move<T, NM, STR>(P, c, -dV, -one, ILc, strip, acc, fm, fe); sm = -fm; FRm += fm; FRe += fe; }
            p.dMR[j * (nr + 1) + i] = sm;
        }
        // right face r_{i+1}
        {
            const T dV = radial_dV<T, UNI>(P, i + 1, j, dt);
            if (!warp_any(nonzero(dV))) {
            } else if (pos(dV)) { move<T, NM, STR>(P, c, dV, -one, ILc, strip, acc, fm, fe); FRm += fm; FRe += fe; }
            else if (neg(dV)) { move<T, NM, STR>(P, c + 1, -dV, one, ILc, strip, acc, fm, fe); FRm -= fm; FRe -= fe; }
            if (i == nr - 1) p.dMR[j * (nr + 1) + nr] = zero;
        }
        // bottom face z_j
        {
            const T dV = vertical_dV<T>(P, i, j, dt);
            T sm = zero;
            if (!warp_any(nonzero(dV))) {
            } else if (pos(dV)) { move<T, NM, STR>(P, c - nr, dV, one, ILc, strip, acc, fm, fe); sm = fm; FZm -= fm; FZe -= fe; }
            else if (neg(dV)) { move<T, NM, STR>(P, c, -dV, -one, ILc, strip, acc, fm, fe); sm = -fm; FZm += fm; FZe += fe; }
            p.dMZ[j * nr + i] = sm;
        }
        // top face z_{j+1}: above the domain only outflow (inflow is void)
        {
            const T dV = vertical_dV<T>(P, i, j + 1, dt);
            T sm = zero;
            if (!warp_any(nonzero(dV))) {
            } else if (pos(dV)) {
                move<T, NM, STR>(P, c, dV, -one, ILc, strip, acc, fm, fe);
                FZm += fm; FZe += fe; sm = fm;
                if (j == nz - 1) t_out += double(fm);
            } else if (neg(dV) && j + 1 < nz) {
                move<T, NM, STR>(P, c + nr, -dV, one, ILc, strip, acc, fm, fe); FZm -= fm; FZe -= fe;
            }
            if (j == nz - 1) p.dMZ[nz * nr + i] = sm;
        }
        // new state in increment form: q' = q^L + (net q-content flux - q^L net carrier
        // flux) / new carrier amount (exact when nothing flows); the energy change is the
        // inflows' (I_donor - I^L) mass, added in FP64
        const T Vc = Geo<T, UNI>::vol(P, i, j);
        T Vm[NM], Mm[NM], rn[NM];
        T MLtot = zero, VLmat = zero, dMtot = zero, dVtot = zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const typename V::T2 fl = p.frL[m][c];
            const T VmL = fl.x * VLc;
            const T MmL = fl.y * VmL;
            MLtot += MmL; VLmat += VmL;
            dMtot += acc.Mm[m]; dVtot += acc.Vm[m];
            Vm[m] = VmL + acc.Vm[m];
            Mm[m] = MmL + acc.Mm[m];
            // nothing moved: the increment (0 - rho^L 0) / V_m is zero (no division)
            const bool moved = nonzero(acc.Mm[m]) || nonzero(acc.Vm[m]);
            rn[m] = !pos(Vm[m]) ? zero : (warp_any(moved) && moved) ? fl.y + (acc.Mm[m] - fl.y * acc.Vm[m]) / Vm[m] : fl.y;
        }
        const T Mtot = MLtot + dMtot, Vtot = VLmat + dVtot;
        double Ic = pos(Mtot) ? ILc : 0.0;
        const bool add_dI = pos(Mtot) && nonzero(acc.dI);
        if (warp_any(add_dI) && add_dI) Ic = ILc + double(acc.dI / Mtot);
        T s0 = zero, s1 = zero, s2 = zero, Dm = zero;
        if (STR && pos(Vtot)) {
            const T iv = one / Vtot;
            const typename V::T2 a = p.sL01[c], b = p.sL2d[c];
            s0 = a.x + (acc.S[0] - a.x * dVtot) * iv;
            s1 = a.y + (acc.S[1] - a.y * dVtot) * iv;
            s2 = b.x + (acc.S[2] - b.x * dVtot) * iv;
            Dm = b.y + (acc.S[3] - b.y * dVtot) * iv;
        }
        T Mkeep = zero, Vkeep = zero, fnew[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            fnew[m] = Vm[m] / Vc;    // a true division: exact 1 for a full resting cell
            if (fnew[m] < P.f_min) {
                if (warp_any(nonzero(Mm[m])) && nonzero(Mm[m])) t_disc += double(Mm[m]);
                Vm[m] = zero;
                Mm[m] = zero;
                rn[m] = zero;
            }
            Mkeep += Mm[m];
            Vkeep += Vm[m];
        }
        if (!pos(Mkeep)) { Ic = 0.0; s0 = s1 = s2 = Dm = zero; }
        T kappa = one;
        const bool inB = j < P.pb, inR = i >= nr - P.pr;
        if (inB || inR) {
            T dsum = zero, phi1 = zero, phi3 = zero;
            if (inB) {
                const T d = p.dB_c[j];
                typename V::T2 a = p.pb_c[c];
                const T rl = one - P.alpha_b * dt;
                a.x = a.x * rl + d * FRm;
                a.y = a.y * rl + d * FRe;
                p.pb_c[c] = a;
                dsum += d; phi1 += a.x; phi3 += a.y;
            }
            if (inR) {
                const int k = j * P.pr + (i - (nr - P.pr));
                const T d = strip_row_c(p, j) ? p.dR_c[i] : zero;
                typename V::T2 a = p.pr_c[k];
                const T rl = one - P.alpha_r * dt;
                a.x = a.x * rl + d * FZm;
                a.y = a.y * rl + d * FZe;
                p.pr_c[k] = a;
                dsum += d; phi1 += a.x; phi3 += a.y;
            }
            if (pos(Mkeep) && pos(dsum)) {
                const T Mref = Vkeep * p.rho_ref[j];
                const T dM = -dt * (dsum * (Mkeep - Mref) + phi1);
                const double dEp = -double(dt) * (double(dsum) * (double(Mkeep) * Ic - double(Mref) * p.I_ref[j]) + double(phi3));
                const T Mnew = Mkeep + dM;
                if (!pos(Mnew)) atomicOr(&p.scal->status, 1);
                t_pml += double(dM);
                kappa = one + dM / Mkeep;
                Ic = Ic + (dEp - Ic * double(dM)) / double(Mnew);
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            if (pos(Vm[m]))
                p.fr[m][c] = V::mk(fnew[m], kappa * rn[m]);
            else
                p.fr[m][c] = V::mk(zero, zero);
        }
        p.I[c] = Ic;
        if (is_nan(Ic)) atomicOr(&p.scal->status, 2);
        if (STR) {
            p.s01[c] = V::mk(s0, s1);
            p.s2d[c] = V::mk(s2, Dm);
        }
    }
    // tallies.  Outflow through the top and the strips' damping happen only in blocks on
    // the top row or in a strip: those sum over the block with one atomic each, when some
    // thread has one.  Elsewhere only the rare clean-up tallies, and a warp that has some
    // adds it by itself, so the block needs no barrier.
    const int bdx = blockDim.x, bdy = blockDim.y;
    const bool edge_block = (by + 1) * bdy > P.nz - 1 || by * bdy < P.pb || (bx + 1) * bdx > nr - P.pr;
    if (!edge_block) {
        if (__any_sync(0xffffffffu, nonzero(t_disc))) {
            const double b_disc = warp_sum(t_disc);
            if ((threadIdx.x & 31) == 0 && b_disc != 0.0) atomicAdd(&p.scal->mass_discarded, b_disc);
        }
    } else if (__syncthreads_or(nonzero(t_out) || nonzero(t_disc) || nonzero(t_pml))) {
        __shared__ double sh[kMaxThreads / 32];
        const double b_out = block_sum(t_out, sh);
        const double b_disc = block_sum(t_disc, sh);
        const double b_pml = block_sum(t_pml, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            if (b_out != 0.0) atomicAdd(&p.scal->mass_out, b_out);
            if (b_disc != 0.0) atomicAdd(&p.scal->mass_discarded, b_disc);
            if (b_pml != 0.0) atomicAdd(&p.scal->mass_pml, b_pml);
        }
    }
}

// ---------------------------------------------------------------------------------
// Phase 3b: momentum remap on the dual grid.
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T dMR_at(const ParamsT<T>& P, int i, int j)
{
    return (j < 0 || j >= P.nz) ? T(0) : P.p.dMR[j * (P.nr + 1) + i];
}
template <typename T>
__device__ __forceinline__ T dMZ_at(const ParamsT<T>& P, int i, int j)
{
    return (i < 0 || i >= P.nr) ? T(0) : P.p.dMZ[j * P.nr + i];
}
// dual mass flux between (i,j) and (i+1,j)
template <typename T>
__device__ __forceinline__ T dual_R(const ParamsT<T>& P, int i, int j)
{
    return T(0.25) * (dMR_at(P, i, j - 1) + dMR_at(P, i + 1, j - 1) + dMR_at(P, i, j) + dMR_at(P, i + 1, j));
}
// dual mass flux between (i,j) and (i,j+1); j == nz: out through the top
template <typename T>
__device__ __forceinline__ T dual_Z(const ParamsT<T>& P, int i, int j)
{
    if (j == P.nz) return T(0.5) * (dMZ_at(P, i - 1, j) + dMZ_at(P, i, j));
    return T(0.25) * (dMZ_at(P, i - 1, j) + dMZ_at(P, i - 1, j + 1) + dMZ_at(P, i, j) + dMZ_at(P, i, j + 1));
}

// The FP64 form shares each dual face between its two vertices (its FP64 pipe is the
// bound, and half the face arithmetic goes); the mixed form, bound by latency, keeps one
// computation per vertex and face and no barrier.
template <typename T> struct ShareFaces { static constexpr bool value = false; };
template <> struct ShareFaces<double> { static constexpr bool value = true; };

// shared memory of phase 3b: the faces to the right and upper neighbours of each thread's
// vertex, 2 x 4 values per thread (FP64 form)
template <typename T>
size_t phase3b_smem(dim3 blk) { return ShareFaces<T>::value ? (size_t)2 * 4 * blk.x * blk.y * sizeof(T) : 0; }

template <typename T>
__device__ __forceinline__ void body_phase3b(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    const T zero = T(0), one = T(1), half = T(0.5);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr, nz = P.nz, nv = nr + 1;
    const PtrsT<T>& p = P.p;
    double t_zmom = 0.0;
    // Each dual face joins two vertices.  Every thread computes the faces to its vertex's
    // right and upper neighbours and leaves them in shared memory; the faces to its left
    // and lower neighbours are those neighbours' (recomputed, identically, on the block's
    // first column and row), so each face is computed once per block.
    constexpr bool share = ShareFaces<T>::value;
    const bool valid = i <= nr && j <= nz;
    const int nt = blockDim.x * blockDim.y, tl = threadIdx.y * blockDim.x + threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem3b[];
    T* sR = reinterpret_cast<T*>(smem3b);
    T* sZ = sR + 4 * nt;
    const int v = j * nv + i;
    typename V::T2 vL = V::mk(zero, zero);
    DualFace<T> oR = {zero, zero, zero, zero}, oZ = {zero, zero, zero, zero};
    if (valid) {
        vL = p.vL[v];
        if (i < nr) {  // face to (i+1, j)
            const T f = dual_R(P, i, j);
            oR = dual_face<T>(f, pos(f) ? vL : p.vL[v + 1]);
        }
        {              // face to (i, j+1), or out through the top
            const T f = dual_Z(P, i, j);
            oZ = dual_face<T>(f, (pos(f) || j == nz) ? vL : p.vL[v + nv]);
        }
    }
    if (share) {
        sR[tl] = oR.f; sR[nt + tl] = oR.fr; sR[2 * nt + tl] = oR.fz; sR[3 * nt + tl] = oR.e;
        sZ[tl] = oZ.f; sZ[nt + tl] = oZ.fr; sZ[2 * nt + tl] = oZ.fz; sZ[3 * nt + tl] = oZ.e;
        __syncthreads();
    }
    if (valid) {
        const T dt = step_dt<T>(p.scal);
        const T m0 = p.mv[v];
        T m = m0, pr = m0 * vL.x, pz = m0 * vL.y;
        T kin = half * m0 * (vL.x * vL.x + vL.y * vL.y);
        DualFace<T> iR = {zero, zero, zero, zero}, iZ = {zero, zero, zero, zero};
        if (i > 0) {   // face to (i-1, j)
            if (share && threadIdx.x > 0) {
                const int k = tl - 1;
                iR = DualFace<T>{sR[k], sR[nt + k], sR[2 * nt + k], sR[3 * nt + k]};
            } else {
                const T f = dual_R(P, i - 1, j);
                iR = dual_face<T>(f, pos(f) ? p.vL[v - 1] : vL);
            }
        }
        if (j > 0) {   // face to (i, j-1)
            if (share && threadIdx.y > 0) {
                const int k = tl - (int)blockDim.x;
                iZ = DualFace<T>{sZ[k], sZ[nt + k], sZ[2 * nt + k], sZ[3 * nt + k]};
            } else {
                const T f = dual_Z(P, i, j - 1);
                iZ = dual_face<T>(f, pos(f) ? p.vL[v - nv] : vL);
            }
        }
        m += iR.f; kin += iR.e;
        m -= oR.f; kin -= oR.e;
        m += iZ.f; kin += iZ.e;
        m -= oZ.f; kin -= oZ.e;
        const T inRr = iR.fr, inRz = iR.fz, outRr = oR.fr, outRz = oR.fz;
        const T inZr = iZ.fr, inZz = iZ.fz, outZr = oZ.fr, outZz = oZ.fz;
        if (warp_any(j == nz) && j == nz) t_zmom += double(outZz);
        pr += (inRr - outRr) + (inZr - outZr);
        pz += (inRz - outRz) + (inZz - outZz);
        // a resting vertex (no momentum, no kinetic energy, no flux, no deficit) gets no heat
        // and, unless a strip's damping gives it momentum below, no velocity: its warp skips
        // the reciprocal and the rest (the results are the same zeros)
        const T dKv = p.dK[v];
        const bool quiet = !nonzero(pr) && !nonzero(pz) && !nonzero(kin) && !nonzero(dKv);
        T kheat = zero, im = zero;
        bool have_im = false;
        if (pos(m) && warp_any(!quiet) && !quiet) {
            im = one / m;
            have_im = true;
            const T dKr = kin - half * (pr * pr + pz * pz) * im;
            kheat = (dKv + dKr) * im;
        }
        p.kheat[v] = kheat;
        T dsum = zero, a2r = zero, a2z = zero;
        if (j < P.pb) {
            const T d = p.dB_v[j];
            typename V::T4 a = p.pb_v[v];
            const T rl = one - P.alpha_b * dt;
            a.x = a.x * rl + d * (outRr - inRr);
            a.y = a.y * rl + d * (outRz - inRz);
            p.pb_v[v] = a;
            dsum += d; a2r += a.x; a2z += a.y;
        }
        if (i > nr - P.pr) {
            const int k = j * P.pr + (i - (nr - P.pr + 1));
            const T d = strip_row_v(p, j, P.nz) ? p.dR_v[i] : zero;
            typename V::T4 a = p.pr_v[k];
            const T rl = one - P.alpha_r * dt;
            a.x = a.x * rl + d * (outZr - inZr);
            a.y = a.y * rl + d * (outZz - inZz);
            p.pr_v[k] = a;
            dsum += d; a2r += a.x; a2z += a.y;
        }
        if (j < P.pb || i > nr - P.pr) {
            pr = pr - dt * (dsum * pr + a2r);
            pz = pz - dt * (dsum * pz + a2z);
        }
        T vr = zero, vz = zero;
        const bool moving = nonzero(pr) || nonzero(pz);
        if (pos(m) && warp_any(moving) && moving) {
            // no material in any adjacent cell after the clean-up: no momentum (the dual
            // mass is then only round-off of the fluxes)
            bool occupied = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int ci = (k == 0 || k == 3) ? i - 1 : i;
                const int cj = (k < 2) ? j - 1 : j;
                if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                for (int mm = 0; mm < P.nmat; ++mm) occupied |= pos(p.fr[mm][cj * nr + ci].x);
            }
            if (occupied) {
                if (!have_im) im = one / m;
                vr = pr * im;
                vz = pz * im;
            }
        }
        if (i == 0 || i == nr) vr = zero;
        if (j == 0) {
            vz = zero;
            if (P.bc_bottom == SALEC_BOTTOM_NOSLIP) vr = zero;
        }
        if (j == nz && P.bc_top == SALEC_TOP_WALL) vz = zero;
        if (is_nan(vr) || is_nan(vz)) atomicOr(&p.scal->status, 2);
        p.v[v] = V::mk(vr, vz);
    }
    // the z-momentum leaving through the top: only blocks on the top vertex row have any
    if ((by + 1) * (int)blockDim.y > nz && __syncthreads_or(nonzero(t_zmom))) {
        __shared__ double sh[kMaxThreads / 32];
        const double b = block_sum(t_zmom, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0 && b != 0.0) atomicAdd(&p.scal->zmom_out, b);
    }
}

// ---------------------------------------------------------------------------------
// Phase 3c: kinetic-energy deficit as heat; advance time.
// ---------------------------------------------------------------------------------
template <typename T, int NM>
__device__ __forceinline__ void body_phase3c(const ParamsT<T>& P, int bx, int by, int gx, int gy)
{
    typedef VT<T> V;
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nr = P.nr, nv = nr + 1;
    const PtrsT<T>& p = P.p;
    if (i < nr && j < P.nz) {
        const int c = j * nr + i;
        T M = T(0);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const typename V::T2 fr = p.fr[m][c];
            M += fr.x * fr.y;
        }
        if (pos(M)) {
            const T add = T(0.25) * (p.kheat[j * nv + i] + p.kheat[j * nv + i + 1] +
                                     p.kheat[(j + 1) * nv + i + 1] + p.kheat[(j + 1) * nv + i]);
            if (warp_any(nonzero(add)) && nonzero(add)) p.I[c] += double(add);
        }
    }
    if (bx == 0 && by == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        DevScalars* s = p.scal;
        s->t += s->dt;
        s->dt_prev = s->dt;
        s->nstep += 1ull;
    }
}

}  // namespace salec
