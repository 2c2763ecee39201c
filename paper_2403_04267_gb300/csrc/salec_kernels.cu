// salec_kernels.cu -- the SALE cycle on sm_103a: one kernel per phase, FP64.
//
//   k_phase0  EoS, tension cut-off, artificial viscosity, Courant dt (block min, then the
//             last block reduces the per-block minima)              Eqs. 1-2, Eq. 14
//   k_phase1  vertex corner forces incl. hoop stress, gravity, PML psi1, v^L, BCs  Eq. 1, Eqs. 16/21
//   k_phase2  swept volumes, strain rates, compatible energy, PML psi2, void/material
//             volume partition, Jaumann + von Mises + damage        Eq. 2, Eqs. 17/22
//   k_phase3a donor-cell VOF remap, clean-up, PML phi1/phi3 + damping   Eqs. 3, 5, 18, 20, 23, 25
//   k_phase3b dual-grid momentum remap, PML phi2 + damping, KE deficit  Eqs. 4, 19, 24
//   k_phase3c kinetic-energy deficit returned as heat; time advance
//
// Layout: cell arrays row-major [j][i] (nr fastest), vertex arrays [j][i] over nr+1;
// paired quantities are double2 so one warp moves 512 contiguous bytes per load.
// Blocks are 32 x 8 threads over (i, j).
#include <cuda_runtime.h>

#include "salec_internal.cuh"

namespace salec {

__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum, result valid in thread 0
__device__ double block_sum(double v, double* sh)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w];
    return s;
}

// ---------------------------------------------------------------------------------
// Phase 0: equation of state, artificial viscosity and the Courant time step.
// ---------------------------------------------------------------------------------
template <int NM, bool STR>
__global__ void __launch_bounds__(kThreads) k_phase0(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr;
    const Ptrs& p = P.p;
    // largest |v| + c of the block; min over cells of dx / (|v| + c) = dx / max(|v| + c)
    // exactly (correctly rounded division is monotonic), so one division per step suffices
    double speed = 0.0;
    if (i < nr && j < P.nz) {
        const int c = j * nr + i;
        double phat = 0.0, phi = 0.0, mass = 0.0, c2m = 0.0, p1 = 0.0, r1 = 0.0;
        const double Ic = p.I[c];
        const double D = STR ? p.s2d[c].y : 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const double2 fr = p.fr[m][c];
            if (pos(fr.x)) {
                double pm, c2;
                eos_eval(P.mat[m], fr.y, Ic, pm, c2);
                const double pmin = (1.0 - D) * P.mat[m].p_t;
                pm = pm < pmin ? pmin : pm;
                phat += fr.x * pm;
                phi += fr.x;
                mass += fr.x * fr.y;
                c2m = max_nonneg(c2m, c2);
                p1 = pm;
                r1 = fr.y;
            }
        }
        double Pc = 0.0, pbar = 0.0;
        if (pos(phi)) {
            const int nv = nr + 1;
            const double2 va = p.v[j * nv + i], vb = p.v[j * nv + i + 1];
            const double2 vc = p.v[(j + 1) * nv + i + 1], vd = p.v[(j + 1) * nv + i];
            const double uL = 0.5 * (va.x + vd.x), uR = 0.5 * (vb.x + vc.x);
            const double uB = 0.5 * (va.y + vb.y), uT = 0.5 * (vd.y + vc.y);
            const double div = (p.A_R[i + 1] * uR - p.A_R[i] * uL + p.A_Z[i] * (uT - uB)) * p.invV[i];
            const double cs = sqrt(c2m);
            // one material: p_bar = p and rho_bar = rho; otherwise divide by Phi once
            const double iphi = NM == 1 ? 1.0 : 1.0 / phi;
            pbar = NM == 1 ? p1 : phat * iphi;
            double q = 0.0;
            if (neg(div)) {
                const double rb = NM == 1 ? r1 : mass * iphi;
                q = rb * (P.cq * P.dx2 * div * div - P.cl * P.dx * cs * div);
            }
            Pc = phat + phi * q;
            const double over = pbar - p.p0[j];
            if (over > p.pmax[c]) p.pmax[c] = over;
            double w = va.x * va.x + va.y * va.y;
            w = max_nonneg(w, vb.x * vb.x + vb.y * vb.y);
            w = max_nonneg(w, vc.x * vc.x + vc.y * vc.y);
            w = max_nonneg(w, vd.x * vd.x + vd.y * vd.y);
            speed = sqrt(w) + cs;
            if (is_nan(speed)) atomicOr(&p.scal->status, 2);
        }
        p.PM[c] = make_double2(Pc, mass * p.V[i]);
        p.pbphi[c] = make_double2(pbar, phi);
    }
    // block maximum (on the bit patterns of the non-negative speeds), then the last block
    // to finish reduces the block maxima
    __shared__ long long sh[kThreads / 32];
    __shared__ bool last;
    const int tid = threadIdx.y * kBlockX + threadIdx.x;
    long long sb = __double_as_longlong(speed);
    for (int o = 16; o > 0; o >>= 1) sb = max(sb, __shfl_down_sync(0xffffffffu, sb, o));
    if ((tid & 31) == 0) sh[tid >> 5] = sb;
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y;
    long long* part = reinterpret_cast<long long*>(p.partial);
    if (tid == 0) {
        long long b = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) b = max(b, sh[w]);
        part[blockIdx.y * gridDim.x + blockIdx.x] = b;
        __threadfence();
        const unsigned prev = atomicAdd(&p.scal->counter, 1u);
        last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    long long m = 0;
    for (int k = tid; k < nblk; k += kThreads) m = max(m, __ldcg(&part[k]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) sh[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        long long b = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) b = max(b, sh[w]);
        DevScalars* s = p.scal;
        double dt = P.growth * s->dt_prev;
        const double cdt = P.cfl * (P.dx / __longlong_as_double(b));
        dt = cdt < dt ? cdt : dt;
        dt = P.dt_max < dt ? P.dt_max : dt;
        if (dt < P.dt_min) s->status |= 4;
        s->dt = dt;
        s->counter = 0u;
    }
}

// ---------------------------------------------------------------------------------
// Phase 1: corner forces, gravity and PML psi1 on the vertices; Lagrangian velocity.
// Cells around vertex (i,j): k = 0 (i-1,j-1) corner c, 1 (i,j-1) corner d,
// 2 (i,j) corner a, 3 (i-1,j) corner b.
// ---------------------------------------------------------------------------------
template <bool STR>
__global__ void __launch_bounds__(kThreads) k_phase1(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    if (i > nr || j > nz) return;
    const Ptrs& p = P.p;
    const double dt = p.scal->dt;
    const int v = j * (nr + 1) + i;
    const double hoop = 0.25 * P.dx2;
    double Pc[4] = {0.0, 0.0, 0.0, 0.0}, Pp[4] = {0.0, 0.0, 0.0, 0.0};
    double devr_rad = 0.0, devz_rad = 0.0, devr_ver = 0.0, devz_ver = 0.0, mass = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ci = (k == 0 || k == 3) ? i - 1 : i;
        const int cj = (k < 2) ? j - 1 : j;
        if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
        const int c = cj * nr + ci;
        const double2 pm = p.PM[c];
        Pc[k] = pm.x;
        mass += 0.25 * pm.y;
        if (STR || P.pr > 0 || P.pb > 0) {
            const double phi = p.pbphi[c].y;
            Pp[k] = pm.x - phi * p.p0[cj];
            if (STR) {
                const double2 s01 = p.s01[c];
                const double srz = p.s2d[c].x;
                const double Srr = phi * s01.x, Szz = phi * s01.y, Srz = phi * srz;
                const double Stt = -(Srr + Szz);
                const double hz = 0.5 * p.A_Z[ci];
                // corner signs: a (k=2), b (k=3) at the bottom of the cell; c (k=0), d (k=1) at the top;
                // a, d on the left face; b, c on the right face
                const double sr = (k == 2 || k == 1) ? 1.0 : -1.0;     // left corners +, right corners -
                const double sz = (k == 2 || k == 3) ? 1.0 : -1.0;     // bottom corners +, top corners -
                devr_rad += sr * hz * Srr - hoop * Stt;
                devz_rad += sr * hz * Srz;
                devr_ver += sz * hz * Srz;
                devz_ver += sz * hz * Szz;
            }
        }
    }
    const double AR = p.A_R[i];
    const double AZl = i > 0 ? p.A_Z[i - 1] : 0.0, AZr = i < nr ? p.A_Z[i] : 0.0;
    const double Fr = 0.5 * AR * (((Pc[0] + Pc[3]) - Pc[1]) - Pc[2]) + (devr_rad + devr_ver);
    const double Fz = 0.5 * (AZl * (Pc[0] - Pc[3]) + AZr * (Pc[1] - Pc[2])) + (devz_rad + devz_ver);
    double psr = 0.0, psz = 0.0;
    if (j < P.pb) {
        const double d = p.dB_v[j];
        double4_32a a = p.pb_v[v];
        const double Tr = 0.5 * AR * (((Pp[0] + Pp[3]) - Pp[1]) - Pp[2]) + devr_rad;
        a.z -= dt * d * Tr;
        a.w -= dt * d * devz_rad;
        p.pb_v[v] = a;
        psr += a.z; psz += a.w;
    }
    if (i > nr - P.pr) {
        const int k = j * P.pr + (i - (nr - P.pr + 1));
        const double d = p.dR_v[i];
        double4_32a a = p.pr_v[k];
        const double Tz = 0.5 * (AZl * (Pp[0] - Pp[3]) + AZr * (Pp[1] - Pp[2])) + devz_ver;
        a.z -= dt * d * devr_ver;
        a.w -= dt * d * Tz;
        p.pr_v[k] = a;
        psr += a.z; psz += a.w;
    }
    const double2 vn = p.v[v];
    double vr = 0.0, vz = 0.0;
    if (pos(mass)) {
        const double im = 1.0 / mass;
        vr = vn.x + dt * ((Fr - psr) * im);
        vz = vn.y + dt * ((Fz - psz) * im - P.g);
    }
    if (i == 0 || i == nr) vr = 0.0;
    if (j == 0) {
        vz = 0.0;
        if (P.bc_bottom == SALEC_BOTTOM_NOSLIP) vr = 0.0;
    }
    if (j == nz && P.bc_top == SALEC_TOP_WALL) vz = 0.0;
    p.vL[v] = make_double2(vr, vz);
    p.mv[v] = mass;
    const double dvr = vr - vn.x, dvz = vz - vn.y;
    p.dK[v] = 0.5 * mass * (dvr * dvr + dvz * dvz);
}

// ---------------------------------------------------------------------------------
// Phase 2: Lagrangian cell update from v^L.
// ---------------------------------------------------------------------------------
template <int NM, bool STR>
__global__ void __launch_bounds__(kThreads) k_phase2(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr;
    if (i >= nr || j >= P.nz) return;
    const Ptrs& p = P.p;
    const int c = j * nr + i;
    const double phi = p.pbphi[c].y;
    if (!pos(phi)) {
#pragma unroll
        for (int m = 0; m < NM; ++m) p.frL[m][c] = make_double2(0.0, 0.0);
        p.VIL[c] = make_double2(p.V[i], 0.0);
        if (STR) { p.sL01[c] = make_double2(0.0, 0.0); p.sL2d[c] = make_double2(0.0, 0.0); }
        return;
    }
    const double dt = p.scal->dt;
    const double dx = P.dx;
    const int nv = nr + 1;
    const double2 va = p.vL[j * nv + i], vb = p.vL[j * nv + i + 1];
    const double2 vc = p.vL[(j + 1) * nv + i + 1], vd = p.vL[(j + 1) * nv + i];
    const double uL = 0.5 * (va.x + vd.x), uR = 0.5 * (vb.x + vc.x);
    const double uB = 0.5 * (va.y + vb.y), uT = 0.5 * (vd.y + vc.y);
    const double idx = 1.0 / dx;
    const double err = (uR - uL) * idx;
    const double ezz = (uT - uB) * idx;
    const double V = p.V[i];
    const double ett = (uR + uL) * p.inv2rc[i];
    const double rad_flux = p.A_R[i + 1] * uR - p.A_R[i] * uL;
    const double ver_flux = p.A_Z[i] * (uT - uB);
    const double dV = dt * (rad_flux + ver_flux);
    const double VL = V + dV;
    const double2 pm = p.PM[c];
    const double Pc = pm.x, M = pm.y;
    double work = 0.0, Pi_rad = -Pc * rad_flux, Pi_ver = -Pc * ver_flux;
    double dvr_dz = 0.0, dvz_dr = 0.0, srr = 0.0, szz = 0.0, srz = 0.0, D = 0.0;
    if (STR) {
        const double2 s01 = p.s01[c], s2d = p.s2d[c];
        srr = s01.x; szz = s01.y; srz = s2d.x; D = s2d.y;
        dvr_dz = 0.5 * ((vd.x + vc.x) - (va.x + vb.x)) * idx;
        dvz_dr = 0.5 * ((vb.y + vc.y) - (va.y + vd.y)) * idx;
        const double Srr = phi * srr, Szz = phi * szz, Srz = phi * srz, Stt = -(Srr + Szz);
        const double erz = 0.5 * (dvr_dz + dvz_dr);
        work = dt * V * (Srr * err + Szz * ezz + Stt * ett + 2.0 * Srz * erz);
        Pi_rad += V * (Srr * err + Stt * ett + Srz * dvz_dr);
        Pi_ver += V * (Szz * ezz + Srz * dvr_dz);
    }
    double psi2 = 0.0;
    if (j < P.pb) {
        double a = p.pb_psi2[c];
        a -= dt * p.dB_c[j] * Pi_rad;
        p.pb_psi2[c] = a;
        psi2 += a;
    }
    if (i >= nr - P.pr) {
        const int k = j * P.pr + (i - (nr - P.pr));
        double a = p.pr_psi2[k];
        a -= dt * p.dR_c[i] * Pi_ver;
        p.pr_psi2[k] = a;
        psi2 += a;
    }
    const double dE = -Pc * dV + work - dt * psi2;
    const double Ic = p.I[c];
    const double IL = pos(M) ? Ic + dE / M : Ic;
    p.VIL[c] = make_double2(VL, IL);
    // volume partition: compression closes void first; expansion shared pro rata with void
    double Vvoid = (1.0 - phi) * V;
    Vvoid = Vvoid < 0.0 ? 0.0 : Vvoid;
    double dVmat;
    if (dV < 0.0) {
        const double dVvoid = dV > -Vvoid ? dV : -Vvoid;
        dVmat = dV - dVvoid;
    } else {
        dVmat = phi * dV;
    }
    bool bad = false;
    double G = 0.0, Y = 0.0, iepsf = 0.0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const double2 fr = p.fr[m][c];
        if (pos(fr.x)) {
            const double Vm = fr.x * V;
            // one material: f_m / Phi = 1; true divisions keep a resting cell exact
            const double VmL = NM == 1 ? Vm + dVmat : Vm + fr.x / phi * dVmat;
            bad |= !pos(VmL);
            p.frL[m][c] = make_double2(VmL / VL, fr.y * (Vm / VmL));
            if (STR && P.mat[m].strength == SALEC_STRENGTH_COLLINS) {
                const Mat& mm = P.mat[m];
                const double pb = p.pbphi[c].x;
                G += fr.x * mm.G;
                Y += fr.x * yield_eval(mm, pb, D);
                double ef = mm.B_dam * (pb - mm.p_bd);
                ef = ef < mm.eps_fb ? mm.eps_fb : ef;
                iepsf += fr.x / ef;
            }
        } else {
            p.frL[m][c] = make_double2(0.0, 0.0);
        }
    }
    if (bad) atomicOr(&p.scal->status, 1);
    if (STR) {
        const double iphi = 1.0 / phi;
        G *= iphi; Y *= iphi; iepsf *= iphi;
        if (pos(G)) {
            const double omega = 0.5 * (dvr_dz - dvz_dr);
            const double erz = 0.5 * (dvr_dz + dvz_dr);
            const double tr3 = (err + ezz + ett) * (1.0 / 3.0);
            const double G2 = 2.0 * G;
            double nrr = srr + dt * (G2 * (err - tr3) + 2.0 * omega * srz);
            double nzz = szz + dt * (G2 * (ezz - tr3) - 2.0 * omega * srz);
            double nrz = srz + dt * (G2 * erz + omega * (szz - srr));
            const double ntt = -(nrr + nzz);
            const double J2 = 0.5 * (nrr * nrr + nzz * nzz + ntt * ntt) + nrz * nrz;
            if (J2 > Y * Y) {
                const double sq = sqrt(J2);
                const double k = Y / sq;
                nrr *= k; nzz *= k; nrz *= k;
                D += (sq - Y) / (1.7320508075688772 * G) * iepsf;
                D = D > 1.0 ? 1.0 : D;
            }
            srr = nrr; szz = nzz; srz = nrz;
        } else {
            srr = 0.0; szz = 0.0; srz = 0.0;
        }
        p.sL01[c] = make_double2(srr, szz);
        p.sL2d[c] = make_double2(srz, D);
    }
}

// ---------------------------------------------------------------------------------
// Phase 3a: donor-cell remap of the cells.
// ---------------------------------------------------------------------------------
template <int NM, bool STR>
struct Acc {
    double Vm[NM], Mm[NM], E, S[4];
};

// Swept volume of the radial face at r_i of row j, and of the vertical face at z_j of
// column i, from the Lagrangian velocities (computed identically by both neighbours).
__device__ __forceinline__ double radial_dV(const Params& P, int i, int j, double dt)
{
    if (i == 0 || i == P.nr) return 0.0;
    const int nv = P.nr + 1;
    const double u = 0.5 * (P.p.vL[j * nv + i].x + P.p.vL[(j + 1) * nv + i].x);
    return dt * P.p.A_R[i] * u;
}
__device__ __forceinline__ double vertical_dV(const Params& P, int i, int j, double dt)
{
    if (j == 0) return 0.0;
    if (j == P.nz && P.bc_top == SALEC_TOP_WALL) return 0.0;
    const int nv = P.nr + 1;
    const double u = 0.5 * (P.p.vL[j * nv + i].y + P.p.vL[j * nv + i + 1].y);
    return dt * P.p.A_Z[i] * u;
}

// Flux of |dV| of the donor cell's Lagrangian contents, added with sign sgn to acc;
// returns the moved mass and energy.
template <int NM, bool STR>
__device__ __forceinline__ void move(const Params& P, int donor, double adV, double sgn, Acc<NM, STR>& acc,
                                     double& mass_out, double& e_out)
{
    const Ptrs& p = P.p;
    double vmat = 0.0, mass = 0.0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const double2 fl = p.frL[m][donor];
        const double dv = adV * fl.x;
        const double dm = fl.y * dv;
        acc.Vm[m] += sgn * dv;
        acc.Mm[m] += sgn * dm;
        vmat += dv;
        mass += dm;
    }
    const double e = p.VIL[donor].y * mass;
    acc.E += sgn * e;
    if (STR) {
        const double2 a = p.sL01[donor], b = p.sL2d[donor];
        acc.S[0] += sgn * (a.x * vmat);
        acc.S[1] += sgn * (a.y * vmat);
        acc.S[2] += sgn * (b.x * vmat);
        acc.S[3] += sgn * (b.y * vmat);
    }
    mass_out = mass;
    e_out = e;
}

template <int NM, bool STR>
__global__ void __launch_bounds__(kThreads) k_phase3a(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    const Ptrs& p = P.p;
    double t_out = 0.0, t_disc = 0.0, t_pml = 0.0;
    if (i < nr && j < nz) {
        const int c = j * nr + i;
        const double dt = p.scal->dt;
        // acc collects the net fluxes; the Lagrangian contents are added back below
        Acc<NM, STR> acc;
        const double2 vil = p.VIL[c];
#pragma unroll
        for (int m = 0; m < NM; ++m) { acc.Vm[m] = 0.0; acc.Mm[m] = 0.0; }
        acc.E = 0.0;
        acc.S[0] = acc.S[1] = acc.S[2] = acc.S[3] = 0.0;
        // net tangential outflows for the PML auxiliaries: radial (bottom strip), vertical (right strip)
        double FRm = 0.0, FRe = 0.0, FZm = 0.0, FZe = 0.0;
        double fm, fe;
        // left face r_i: positive dV flows from (i-1,j) into this cell
        {
            const double dV = radial_dV(P, i, j, dt);
            double sm = 0.0;
            if (pos(dV)) { move<NM, STR>(P, c - 1, dV, 1.0, acc, fm, fe); sm = fm; FRm -= fm; FRe -= fe; }
            else if (neg(dV)) { move<NM, STR>(P, c, -dV, -1.0, acc, fm, fe); sm = -fm; FRm += fm; FRe += fe; }
            p.dMR[j * (nr + 1) + i] = sm;
        }
        // right face r_{i+1}
        {
            const double dV = radial_dV(P, i + 1, j, dt);
            if (pos(dV)) { move<NM, STR>(P, c, dV, -1.0, acc, fm, fe); FRm += fm; FRe += fe; }
            else if (neg(dV)) { move<NM, STR>(P, c + 1, -dV, 1.0, acc, fm, fe); FRm -= fm; FRe -= fe; }
            if (i == nr - 1) p.dMR[j * (nr + 1) + nr] = 0.0;
        }
        // bottom face z_j
        {
            const double dV = vertical_dV(P, i, j, dt);
            double sm = 0.0;
            if (pos(dV)) { move<NM, STR>(P, c - nr, dV, 1.0, acc, fm, fe); sm = fm; FZm -= fm; FZe -= fe; }
            else if (neg(dV)) { move<NM, STR>(P, c, -dV, -1.0, acc, fm, fe); sm = -fm; FZm += fm; FZe += fe; }
            p.dMZ[j * nr + i] = sm;
        }
        // top face z_{j+1}: above the domain only outflow (inflow is void)
        {
            const double dV = vertical_dV(P, i, j + 1, dt);
            double sm = 0.0;
            if (pos(dV)) {
                move<NM, STR>(P, c, dV, -1.0, acc, fm, fe);
                FZm += fm; FZe += fe; sm = fm;
                if (j == nz - 1) t_out += fm;
            } else if (neg(dV) && j + 1 < nz) {
                move<NM, STR>(P, c + nr, -dV, 1.0, acc, fm, fe); FZm -= fm; FZe -= fe;
            }
            if (j == nz - 1) p.dMZ[nz * nr + i] = sm;
        }
        // new state in increment form: q' = q^L + (net q-content flux - q^L net carrier
        // flux) / new carrier amount (exact when nothing flows)
        const double V = p.V[i];
        double Vm[NM], Mm[NM], rn[NM];
        double MLtot = 0.0, VLmat = 0.0, dMtot = 0.0, dVtot = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const double2 fl = p.frL[m][c];
            const double VmL = fl.x * vil.x;
            const double MmL = fl.y * VmL;
            MLtot += MmL; VLmat += VmL;
            dMtot += acc.Mm[m]; dVtot += acc.Vm[m];
            Vm[m] = VmL + acc.Vm[m];
            Mm[m] = MmL + acc.Mm[m];
            rn[m] = pos(Vm[m]) ? fl.y + (acc.Mm[m] - fl.y * acc.Vm[m]) / Vm[m] : 0.0;
        }
        const double Mtot = MLtot + dMtot, Vtot = VLmat + dVtot;
        double Ic = pos(Mtot) ? vil.y + (acc.E - vil.y * dMtot) / Mtot : 0.0;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, Dm = 0.0;
        if (STR && pos(Vtot)) {
            const double iv = 1.0 / Vtot;
            const double2 a = p.sL01[c], b = p.sL2d[c];
            s0 = a.x + (acc.S[0] - a.x * dVtot) * iv;
            s1 = a.y + (acc.S[1] - a.y * dVtot) * iv;
            s2 = b.x + (acc.S[2] - b.x * dVtot) * iv;
            Dm = b.y + (acc.S[3] - b.y * dVtot) * iv;
        }
        double Mkeep = 0.0, Vkeep = 0.0, fnew[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            fnew[m] = Vm[m] / V;    // a true division: exact 1 for a full resting cell
            if (fnew[m] < P.f_min) {
                t_disc += Mm[m];
                Vm[m] = 0.0;
                Mm[m] = 0.0;
                rn[m] = 0.0;
            }
            Mkeep += Mm[m];
            Vkeep += Vm[m];
        }
        if (!pos(Mkeep)) { Ic = 0.0; s0 = s1 = s2 = Dm = 0.0; }
        double kappa = 1.0;
        const bool inB = j < P.pb, inR = i >= nr - P.pr;
        if (inB || inR) {
            double dsum = 0.0, phi1 = 0.0, phi3 = 0.0;
            if (inB) {
                const double d = p.dB_c[j];
                double2 a = p.pb_c[c];
                a.x += d * FRm;
                a.y += d * FRe;
                p.pb_c[c] = a;
                dsum += d; phi1 += a.x; phi3 += a.y;
            }
            if (inR) {
                const int k = j * P.pr + (i - (nr - P.pr));
                const double d = p.dR_c[i];
                double2 a = p.pr_c[k];
                a.x += d * FZm;
                a.y += d * FZe;
                p.pr_c[k] = a;
                dsum += d; phi1 += a.x; phi3 += a.y;
            }
            if (pos(Mkeep) && pos(dsum)) {
                const double Mref = Vkeep * p.rho_ref[j];
                const double dM = -dt * (dsum * (Mkeep - Mref) + phi1);
                const double dEp = -dt * (dsum * (Mkeep * Ic - Mref * p.I_ref[j]) + phi3);
                const double Mnew = Mkeep + dM;
                if (!(Mnew > 0.0)) atomicOr(&p.scal->status, 1);
                t_pml += dM;
                kappa = 1.0 + dM / Mkeep;
                Ic = Ic + (dEp - Ic * dM) / Mnew;
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            if (pos(Vm[m]))
                p.fr[m][c] = make_double2(fnew[m], kappa * rn[m]);
            else
                p.fr[m][c] = make_double2(0.0, 0.0);
        }
        p.I[c] = Ic;
        if (Ic != Ic) atomicOr(&p.scal->status, 2);
        if (STR) {
            p.s01[c] = make_double2(s0, s1);
            p.s2d[c] = make_double2(s2, Dm);
        }
        (void)V;
    }
    // tallies: block sums, one atomic per block
    __shared__ double sh[kThreads / 32];
    const double b_out = block_sum(t_out, sh);
    const double b_disc = block_sum(t_disc, sh);
    const double b_pml = block_sum(t_pml, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        if (b_out != 0.0) atomicAdd(&p.scal->mass_out, b_out);
        if (b_disc != 0.0) atomicAdd(&p.scal->mass_discarded, b_disc);
        if (b_pml != 0.0) atomicAdd(&p.scal->mass_pml, b_pml);
    }
}

// ---------------------------------------------------------------------------------
// Phase 3b: momentum remap on the dual grid.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double dMR_at(const Params& P, int i, int j)
{
    return (j < 0 || j >= P.nz) ? 0.0 : P.p.dMR[j * (P.nr + 1) + i];
}
__device__ __forceinline__ double dMZ_at(const Params& P, int i, int j)
{
    return (i < 0 || i >= P.nr) ? 0.0 : P.p.dMZ[j * P.nr + i];
}
// dual mass flux between (i,j) and (i+1,j)
__device__ __forceinline__ double dual_R(const Params& P, int i, int j)
{
    return 0.25 * (dMR_at(P, i, j - 1) + dMR_at(P, i + 1, j - 1) + dMR_at(P, i, j) + dMR_at(P, i + 1, j));
}
// dual mass flux between (i,j) and (i,j+1); j == nz: out through the top
__device__ __forceinline__ double dual_Z(const Params& P, int i, int j)
{
    if (j == P.nz) return 0.5 * (dMZ_at(P, i - 1, j) + dMZ_at(P, i, j));
    return 0.25 * (dMZ_at(P, i - 1, j) + dMZ_at(P, i - 1, j + 1) + dMZ_at(P, i, j) + dMZ_at(P, i, j + 1));
}

__global__ void __launch_bounds__(kThreads) k_phase3b(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr, nz = P.nz, nv = nr + 1;
    const Ptrs& p = P.p;
    double t_zmom = 0.0;
    if (i <= nr && j <= nz) {
        const int v = j * nv + i;
        const double dt = p.scal->dt;
        const double2 vL = p.vL[v];
        const double m0 = p.mv[v];
        double m = m0, pr = m0 * vL.x, pz = m0 * vL.y;
        double kin = 0.5 * m0 * (vL.x * vL.x + vL.y * vL.y);
        double outRr = 0.0, outRz = 0.0, inRr = 0.0, inRz = 0.0;
        double outZr = 0.0, outZz = 0.0, inZr = 0.0, inZz = 0.0;
        if (i > 0) {   // face to (i-1, j)
            const double f = dual_R(P, i - 1, j);
            const double2 w = pos(f) ? p.vL[v - 1] : vL;
            inRr = f * w.x; inRz = f * w.y;
            m += f; kin += 0.5 * f * (w.x * w.x + w.y * w.y);
        }
        if (i < nr) {  // face to (i+1, j)
            const double f = dual_R(P, i, j);
            const double2 w = pos(f) ? vL : p.vL[v + 1];
            outRr = f * w.x; outRz = f * w.y;
            m -= f; kin -= 0.5 * f * (w.x * w.x + w.y * w.y);
        }
        if (j > 0) {   // face to (i, j-1)
            const double f = dual_Z(P, i, j - 1);
            const double2 w = pos(f) ? p.vL[v - nv] : vL;
            inZr = f * w.x; inZz = f * w.y;
            m += f; kin += 0.5 * f * (w.x * w.x + w.y * w.y);
        }
        {              // face to (i, j+1), or out through the top
            const double f = dual_Z(P, i, j);
            const double2 w = (pos(f) || j == nz) ? vL : p.vL[v + nv];
            outZr = f * w.x; outZz = f * w.y;
            m -= f; kin -= 0.5 * f * (w.x * w.x + w.y * w.y);
            if (j == nz) t_zmom += outZz;
        }
        pr += (inRr - outRr) + (inZr - outZr);
        pz += (inRz - outRz) + (inZz - outZz);
        double kheat = 0.0, im = 0.0;
        if (pos(m)) {
            im = 1.0 / m;
            const double dKr = kin - 0.5 * (pr * pr + pz * pz) * im;
            kheat = (p.dK[v] + dKr) * im;
        }
        p.kheat[v] = kheat;
        double dsum = 0.0, a2r = 0.0, a2z = 0.0;
        if (j < P.pb) {
            const double d = p.dB_v[j];
            double4_32a a = p.pb_v[v];
            a.x += d * (outRr - inRr);
            a.y += d * (outRz - inRz);
            p.pb_v[v] = a;
            dsum += d; a2r += a.x; a2z += a.y;
        }
        if (i > nr - P.pr) {
            const int k = j * P.pr + (i - (nr - P.pr + 1));
            const double d = p.dR_v[i];
            double4_32a a = p.pr_v[k];
            a.x += d * (outZr - inZr);
            a.y += d * (outZz - inZz);
            p.pr_v[k] = a;
            dsum += d; a2r += a.x; a2z += a.y;
        }
        if (j < P.pb || i > nr - P.pr) {
            pr = pr - dt * (dsum * pr + a2r);
            pz = pz - dt * (dsum * pz + a2z);
        }
        // no material in any adjacent cell after the clean-up: no momentum (the dual mass
        // is then only round-off of the fluxes)
        bool occupied = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ci = (k == 0 || k == 3) ? i - 1 : i;
            const int cj = (k < 2) ? j - 1 : j;
            if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
            for (int mm = 0; mm < P.nmat; ++mm) occupied |= pos(p.fr[mm][cj * nr + ci].x);
        }
        double vr = 0.0, vz = 0.0;
        if (pos(m) && occupied) { vr = pr * im; vz = pz * im; }
        if (i == 0 || i == nr) vr = 0.0;
        if (j == 0) {
            vz = 0.0;
            if (P.bc_bottom == SALEC_BOTTOM_NOSLIP) vr = 0.0;
        }
        if (j == nz && P.bc_top == SALEC_TOP_WALL) vz = 0.0;
        if (is_nan(vr) || is_nan(vz)) atomicOr(&p.scal->status, 2);
        p.v[v] = make_double2(vr, vz);
    }
    __shared__ double sh[kThreads / 32];
    const double b = block_sum(t_zmom, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0 && b != 0.0) atomicAdd(&p.scal->zmom_out, b);
}

// ---------------------------------------------------------------------------------
// Phase 3c: kinetic-energy deficit as heat; advance time.
// ---------------------------------------------------------------------------------
template <int NM>
__global__ void __launch_bounds__(kThreads) k_phase3c(Params P)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr, nv = nr + 1;
    const Ptrs& p = P.p;
    if (i < nr && j < P.nz) {
        const int c = j * nr + i;
        double M = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const double2 fr = p.fr[m][c];
            M += fr.x * fr.y;
        }
        if (pos(M)) {
            const double add = 0.25 * (p.kheat[j * nv + i] + p.kheat[j * nv + i + 1] +
                                       p.kheat[(j + 1) * nv + i + 1] + p.kheat[(j + 1) * nv + i]);
            p.I[c] += add;
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        DevScalars* s = p.scal;
        s->t += s->dt;
        s->dt_prev = s->dt;
        s->nstep += 1ull;
    }
}

// ---------------------------------------------------------------------------------
// Read-out kernels
// ---------------------------------------------------------------------------------
template <int NM>
__global__ void __launch_bounds__(kThreads) k_pressure(Params P, double* out)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    if (i >= P.nr || j >= P.nz) return;
    const int c = j * P.nr + i;
    const Ptrs& p = P.p;
    const double D = P.any_strength ? p.s2d[c].y : 0.0;
    double phat = 0.0, phi = 0.0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const double2 fr = p.fr[m][c];
        if (fr.x > 0.0) {
            double pm, c2;
            eos_eval(P.mat[m], fr.y, p.I[c], pm, c2);
            const double pmin = (1.0 - D) * P.mat[m].p_t;
            pm = pm < pmin ? pmin : pm;
            phat += fr.x * pm;
            phi += fr.x;
        }
    }
    out[c] = phi > 0.0 ? phat / phi : 0.0;
}

// one thread per column: scan down from the top for sum_m f_m >= 1/2
template <int NM>
__global__ void k_column_heights(Params P, double* h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nr) return;
    const int nr = P.nr, nz = P.nz;
    const double dx = P.dx;
    auto phi_at = [&](int j) {
        double f = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) f += P.p.fr[m][j * nr + i].x;
        return f;
    };
    double out = 0.0;
    double up = 0.0;
    for (int j = nz - 1; j >= 0; --j) {
        const double phi = phi_at(j);
        if (phi >= 0.5) {
            const double zc = (j + 0.5) * dx;
            out = (j == nz - 1) ? zc : zc + (phi - 0.5) / (phi - up) * dx;
            break;
        }
        up = phi;
    }
    h[i] = out;
}

// per-block sums of mass, z-momentum, kinetic and internal energy
template <int NM>
__global__ void __launch_bounds__(kThreads) k_conservation(Params P, double* partial4)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nr = P.nr, nz = P.nz;
    const Ptrs& p = P.p;
    auto cmass = [&](int ci, int cj) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const double2 fr = p.fr[m][cj * nr + ci];
            s += fr.x * fr.y;
        }
        return s * p.V[ci];
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
        const double2 vv = p.v[j * (nr + 1) + i];
        pz = m * vv.y;
        ke = 0.5 * m * (vv.x * vv.x + vv.y * vv.y);
    }
    __shared__ double sh[kThreads / 32];
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
static dim3 cell_grid(int nr, int nz) { return dim3((nr + kBlockX - 1) / kBlockX, (nz + kBlockY - 1) / kBlockY); }
static dim3 vert_grid(int nr, int nz) { return dim3((nr + 1 + kBlockX - 1) / kBlockX, (nz + 1 + kBlockY - 1) / kBlockY); }

int cell_blocks(int nr, int nz) { dim3 g = cell_grid(nr, nz); return (int)(g.x * g.y); }
int vertex_blocks(int nr, int nz) { dim3 g = vert_grid(nr, nz); return (int)(g.x * g.y); }
int launches_per_step() { return 6; }

const char* kernel_name(int k)
{
    static const char* names[] = {"k_phase0", "k_phase1", "k_phase2", "k_phase3a", "k_phase3b", "k_phase3c"};
    return (k >= 0 && k < 6) ? names[k] : "";
}

// One cycle; with ev != nullptr an event is recorded before the first kernel and after
// each kernel (7 events) so per-kernel durations can be read later on the same stream.
template <int NM, bool STR>
static cudaError_t step_impl(const Params& P, cudaStream_t s, cudaEvent_t* ev)
{
    const dim3 blk(kBlockX, kBlockY);
    const dim3 gc = cell_grid(P.nr, P.nz), gv = vert_grid(P.nr, P.nz);
    if (ev) cudaEventRecord(ev[0], s);
    k_phase0<NM, STR><<<gc, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[1], s);
    k_phase1<STR><<<gv, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[2], s);
    k_phase2<NM, STR><<<gc, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[3], s);
    k_phase3a<NM, STR><<<gc, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[4], s);
    k_phase3b<<<gv, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[5], s);
    k_phase3c<NM><<<gc, blk, 0, s>>>(P);
    if (ev) cudaEventRecord(ev[6], s);
    return cudaGetLastError();
}

cudaError_t launch_step(const Params& P, cudaStream_t s, cudaEvent_t* ev)
{
    const bool st = P.any_strength != 0;
    switch (P.nmat) {
    case 1: return st ? step_impl<1, true>(P, s, ev) : step_impl<1, false>(P, s, ev);
    case 2: return st ? step_impl<2, true>(P, s, ev) : step_impl<2, false>(P, s, ev);
    case 3: return st ? step_impl<3, true>(P, s, ev) : step_impl<3, false>(P, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pressure(const Params& P, double* out, cudaStream_t s)
{
    const dim3 blk(kBlockX, kBlockY), g = cell_grid(P.nr, P.nz);
    switch (P.nmat) {
    case 1: k_pressure<1><<<g, blk, 0, s>>>(P, out); break;
    case 2: k_pressure<2><<<g, blk, 0, s>>>(P, out); break;
    case 3: k_pressure<3><<<g, blk, 0, s>>>(P, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_column_heights(const Params& P, double* h, cudaStream_t s)
{
    const int t = 128, b = (P.nr + t - 1) / t;
    switch (P.nmat) {
    case 1: k_column_heights<1><<<b, t, 0, s>>>(P, h); break;
    case 2: k_column_heights<2><<<b, t, 0, s>>>(P, h); break;
    case 3: k_column_heights<3><<<b, t, 0, s>>>(P, h); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_conservation(const Params& P, double* partial4, int* nblocks, cudaStream_t s)
{
    const dim3 blk(kBlockX, kBlockY), g = vert_grid(P.nr, P.nz);
    *nblocks = (int)(g.x * g.y);
    switch (P.nmat) {
    case 1: k_conservation<1><<<g, blk, 0, s>>>(P, partial4); break;
    case 2: k_conservation<2><<<g, blk, 0, s>>>(P, partial4); break;
    case 3: k_conservation<3><<<g, blk, 0, s>>>(P, partial4); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace salec
