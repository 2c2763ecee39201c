// salec_fused.cu -- the whole SALE cycle (Fig. 1a of the paper: Lagrangian step, then
// Eulerian step) in one kernel per step.
//
// Each CTA owns a TW x TH tile of cells (and the vertices at their lower-left corners;
// the last tile of a row or column also owns the vertices on the grid's far edge).  It
// stages the state of the tile and a halo of H = 3 cells around it in shared memory and
// runs the phases on regions that shrink by one cell or vertex per dependency:
//   phase 0  EoS, tension cut-off, artificial viscosity   cells    [-3, T+3)
//   phase 1  corner forces, PML psi1, v^L                  vertices [-2, T+3)
//   phase 2  energy, volume partition, strength, psi2      cells    [-2, T+2)
//   phase 3a donor-cell remap, clean-up, phi1/phi3         cells    [-1, T+1)
//   phase 3b dual-grid momentum remap, phi2                vertices [ 0, T+1)
//   phase 3c kinetic-energy deficit as heat                cells    [ 0, T)
// and then forms, for its own cells, the Courant rate of the new state (Eq. 14): the next
// step's time step comes from the running maximum over all tiles, which a one-thread
// kernel turns into dt before the next step starts.  Halo cells are computed by every
// tile that needs them, from the same inputs with the same arithmetic as the phase
// kernels, so the tiles agree on them; only the owner writes a result.  Since a tile reads
// its neighbours' cells, the fields the step rewrites (fractions and densities, energy,
// stress and damage, velocities, PML auxiliaries) are read from one copy and written to
// another (ping-pong); the peak over-pressure is read and written by its owner only and
// stays in place.  Per step the grid's state is read once (plus the halo) and written
// once; the phase kernels' intermediates (pressures, Lagrangian state, face fluxes,
// vertex masses) never leave the SM.
#include <cuda_runtime.h>

#include "salec_device.cuh"
#include "salec_tma.cuh"

namespace salec {

namespace {

constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Shared-memory plan of a tile: arrays that live through the whole cycle, then the inputs
// and phase-0 results (dead after phase 2), overlaid by the remap's results.
template <typename T, int NM, bool STR, int TW, int TH>
struct TileLayout {
    typedef typename VT<T>::T2 T2;
    static constexpr int H = 3;
    static constexpr int CW = TW + 2 * H, CH = TH + 2 * H;   // cell frame
    static constexpr int VW = CW + 1, VH = CH + 1;           // vertex frame
    static constexpr int NC = CW * CH, NV = VW * VH;
    static constexpr bool PBPHI = NM > 1 || STR;              // keep (p_bar, Phi) per cell
    static constexpr size_t c2 = al16(NC * sizeof(T2)), c1 = al16(NC * sizeof(T)), cd = al16(NC * sizeof(double));
    static constexpr size_t v2 = al16(NV * sizeof(T2)), v1 = al16(NV * sizeof(T));
    // whole cycle
    static constexpr size_t o_vL = 0;
    static constexpr size_t o_mv = o_vL + v2;
    static constexpr size_t o_dK = o_mv + v1;
    static constexpr size_t o_frL = o_dK + v1;
    static constexpr size_t o_VL = o_frL + NM * c2;
    static constexpr size_t o_IL = o_VL + c1;
    static constexpr size_t o_sL = o_IL + cd;
    static constexpr size_t o_red = o_sL + (STR ? 2 * c2 : 0);
    static constexpr size_t o_early = o_red + al16(32 * 5 * sizeof(double));
    // inputs and phase 0
    static constexpr size_t o_vo = o_early;
    static constexpr size_t o_fro = o_vo + v2;
    static constexpr size_t o_Io = o_fro + NM * c2;
    static constexpr size_t o_PM = o_Io + cd;
    static constexpr size_t o_pbphi = o_PM + c2;
    static constexpr size_t o_so = o_pbphi + (PBPHI ? c2 : 0);
    static constexpr size_t early_end = o_so + (STR ? 2 * c2 : 0);
    // remap results, over the inputs
    static constexpr size_t o_dMR = o_early;
    static constexpr size_t o_dMZ = o_dMR + al16(VW * CH * sizeof(T));
    static constexpr size_t o_frn = o_dMZ + al16(CW * VH * sizeof(T));
    static constexpr size_t o_In = o_frn + NM * c2;
    static constexpr size_t o_kheat = o_In + cd;
    static constexpr size_t o_vn = o_kheat + v1;
    static constexpr size_t o_Dn = o_vn + v2;
    static constexpr size_t late_end = o_Dn + (STR ? c1 : 0);
    static constexpr size_t bytes = early_end > late_end ? early_end : late_end;
};

// Tile shape, threads and minimum resident CTAs per SM of an instantiation: the mixed form
// of one hydrodynamic material takes 32 x 32 cells (two CTAs of 105 KB per SM); the other
// forms 32 x 16.
template <typename T, int NM, bool STR>
struct TileShape {
    static constexpr bool big = sizeof(T) == 4 && NM == 1 && !STR;
    static constexpr int TW = 32, TH = big ? 32 : 16, NT = 512;
    // two CTAs per SM (64 registers a thread) where two plans fit the SM's 228 KB of
    // shared memory in the mixed form; otherwise one (the FP64 form keeps 128 registers)
    static constexpr size_t bytes = TileLayout<T, NM, STR, TW, TH>::bytes;
    static constexpr int MINB = (sizeof(T) == 4 && 2 * (bytes + 1024) <= 228 * 1024) ? 2 : 1;
};

// What one donor moves through a face: its Lagrangian contents in proportion |dV| / V^L
// (the phase-3a rule), read from the tile's shared memory.
template <typename T, int NM, bool STR>
struct TileDonor {
    typedef typename VT<T>::T2 T2;
    const T2* frL[NM];
    const double* IL;
    const T2* sL01;
    const T2* sL2d;
};

template <typename T, int NM, bool STR>
__device__ __forceinline__ void move_s(const TileDonor<T, NM, STR>& d, int donor, T adV, T sgn, double Iself, bool strip,
                                       Acc<T, NM>& acc, T& mass_out, T& e_out)
{
    typedef typename VT<T>::T2 T2;
    T vmat = T(0), mass = T(0);
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const T2 fl = d.frL[m][donor];
        const T dv = adV * fl.x;
        const T dm = fl.y * dv;
        acc.Vm[m] += sgn * dv;
        acc.Mm[m] += sgn * dm;
        vmat += dv;
        mass += dm;
    }
    const double Id = d.IL[donor];
    if (pos(sgn)) acc.dI += T(Id - Iself) * mass;
    if (STR) {
        const T2 a = d.sL01[donor], b = d.sL2d[donor];
        acc.S[0] += sgn * (a.x * vmat);
        acc.S[1] += sgn * (a.y * vmat);
        acc.S[2] += sgn * (b.x * vmat);
        acc.S[3] += sgn * (b.y * vmat);
    }
    mass_out = mass;
    e_out = strip ? T(Id) * mass : T(0);
}

// Asynchronous copy of N bytes (4, 8 or 16) from global to shared memory without a round
// trip through registers (so every load of the frame is in flight at once); with
// valid == false the destination is zero-filled and nothing is read (src must still be a
// valid address).  Completed by cp_async_wait() before the barrier that publishes them.
template <int N>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int sz = valid ? N : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(N), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// store the upper or lower pair of a strip vertex's four auxiliaries (phi2 r, z | psi1 r, z)
template <typename T4, typename T2>
__device__ __forceinline__ void store_pair(T4* a, int half, T2 v) { reinterpret_cast<T2*>(a)[half] = v; }

}  // namespace

// Registers a thread of the tile kernel may take: what its occupancy leaves (65536 per SM),
// or REGS where that is set (the instantiation that runs beside the copy kernel keeps 120
// of its 128, so that its 16 warps leave room on the SM for the copy warp).
template <int NT, int MINB, int REGS>
struct TileRegs {
    static constexpr int all = 65536 / (NT * MINB);
    static constexpr int value = REGS ? REGS : (all > 255 ? 255 : all);
};

template <typename T, int NM, bool STR, bool UNI, int TW, int TH, int NT, int MINB, int REGS = 0>
__global__ void __launch_bounds__(NT, MINB) __maxnreg__((TileRegs<NT, MINB, REGS>::value))
    k_step_fused(const ParamsT<T> P, const OutPtrsT<T> O)
{
    typedef VT<T> V;
    typedef typename V::T2 T2;
    typedef typename V::T4 T4;
    typedef Geo<T, UNI> GE;
    typedef TileLayout<T, NM, STR, TW, TH> L;
    constexpr int H = L::H, CW = L::CW, CH = L::CH, VW = L::VW, NC = L::NC, NV = L::NV;
    constexpr bool PBPHI = L::PBPHI;
    extern __shared__ __align__(16) unsigned char smem[];
    T2* s_vL = reinterpret_cast<T2*>(smem + L::o_vL);
    T* s_mv = reinterpret_cast<T*>(smem + L::o_mv);
    T* s_dK = reinterpret_cast<T*>(smem + L::o_dK);
    T2* s_frL[NM];
    T2* s_fro[NM];
    T2* s_frn[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        s_frL[m] = reinterpret_cast<T2*>(smem + L::o_frL + m * L::c2);
        s_fro[m] = reinterpret_cast<T2*>(smem + L::o_fro + m * L::c2);
        s_frn[m] = reinterpret_cast<T2*>(smem + L::o_frn + m * L::c2);
    }
    T* s_VL = reinterpret_cast<T*>(smem + L::o_VL);
    double* s_IL = reinterpret_cast<double*>(smem + L::o_IL);
    T2* s_sL01 = reinterpret_cast<T2*>(smem + L::o_sL);
    T2* s_sL2d = reinterpret_cast<T2*>(smem + L::o_sL + L::c2);
    double* s_red = reinterpret_cast<double*>(smem + L::o_red);
    T2* s_vo = reinterpret_cast<T2*>(smem + L::o_vo);
    double* s_Io = reinterpret_cast<double*>(smem + L::o_Io);
    T2* s_PM = reinterpret_cast<T2*>(smem + L::o_PM);
    T2* s_pbphi = reinterpret_cast<T2*>(smem + L::o_pbphi);
    T2* s_so01 = reinterpret_cast<T2*>(smem + L::o_so);
    T2* s_so2d = reinterpret_cast<T2*>(smem + L::o_so + L::c2);
    T* s_dMR = reinterpret_cast<T*>(smem + L::o_dMR);
    T* s_dMZ = reinterpret_cast<T*>(smem + L::o_dMZ);
    double* s_In = reinterpret_cast<double*>(smem + L::o_In);
    T* s_kheat = reinterpret_cast<T*>(smem + L::o_kheat);
    T2* s_vn = reinterpret_cast<T2*>(smem + L::o_vn);
    T* s_Dn = reinterpret_cast<T*>(smem + L::o_Dn);

    const T zero = T(0), one = T(1), half = T(0.5), two = T(2);
    const PtrsT<T>& p = P.p;
    const int nr = P.nr, nz = P.nz, nv = nr + 1;
    const int tid = threadIdx.x;
    const int nbx = (nr + TW - 1) / TW, nby = (nz + TH - 1) / TH;
    const T dt = step_dt<T>(p.scal);
    double t_out = 0.0, t_disc = 0.0, t_pml = 0.0, t_zmom = 0.0;
    T speed_max = zero;
    // The CTA takes tiles from the queue the rest-tile kernel filled (complete: that kernel
    // ran before this one) until it is empty, the front of the list first, then the back
    // from its end; the tallies and the Courant maximum collect over all of them.
    __shared__ int s_tile;
    const int nfront = min(O.work->count, nbx * nby), queued = min(nfront + O.work->back, nbx * nby);
    for (;;) {
    if (tid == 0) {
        const int t = atomicAdd(&O.work->next, 1);
        s_tile = t < nfront ? O.list[t] : t < queued ? O.list[nbx * nby - 1 - (t - nfront)] : -1;
    }
    __syncthreads();        // also: every thread is done with the previous tile's shared memory
    const int tile = s_tile;
    if (tile < 0) break;
    const int bx = tile % nbx, by = tile / nbx;
    const int ox = bx * TW, oy = by * TH;
    const int x0 = ox - H, y0 = oy - H;            // grid indices of frame position 0
    const bool last_x = bx == nbx - 1, last_y = by == nby - 1;

    // ---- stage the state of the frame (cells and vertices outside the grid read as empty):
    // asynchronous copies, all in flight together
    for (int k = tid; k < NV; k += NT) {
        const int i = x0 + k % VW, j = y0 + k / VW;
        const bool in = i >= 0 && i <= nr && j >= 0 && j <= nz;
        cp_async<sizeof(T2)>(&s_vo[k], in ? &p.v[j * nv + i] : p.v, in);
    }
    for (int k = tid; k < NC; k += NT) {
        const int i = x0 + k % CW, j = y0 + k / CW;
        const bool in = i >= 0 && i < nr && j >= 0 && j < nz;
        const int c = in ? j * nr + i : 0;
#pragma unroll
        for (int m = 0; m < NM; ++m) cp_async<sizeof(T2)>(&s_fro[m][k], &p.fr[m][c], in);
        cp_async<8>(&s_Io[k], &p.I[c], in);
        cp_async<sizeof(T2)>(&s_PM[k], &p.eosc[c], in);
        if (STR) {
            cp_async<sizeof(T2)>(&s_so01[k], &p.s01[c], in);
            cp_async<sizeof(T2)>(&s_so2d[k], &p.s2d[c], in);
        }
    }
    cp_async_wait();
    __syncthreads();

    // ---- a quiescent frame: every vertex at rest, every material fraction exactly 0 or 1,
    // zero pressure in the equation-of-state cache (so no viscosity either: div v = 0), no
    // deviatoric stress, no gravity, no absorbing strip in the frame.  Then every phase
    // returns its input: zero forces leave v^L = v = 0, no volume changes (V_m^L / V^L =
    // V / V = 1 for a full cell), no face carries anything, nothing is heated; the own cells'
    // outputs are their inputs (an empty cell's as zeros, as the remap writes it), the peak
    // over-pressure update is the same, the Courant rate is c / L.  The tile then only
    // reads and writes its state.
    bool quiet = !nonzero(P.g) && y0 >= P.pb && x0 + CW <= nr - P.pr;
    if (quiet) {
        bool q = true;
        for (int k = tid; k < NV; k += NT) {
            const T2 v = s_vo[k];
            q = q && !nonzero(v.x) && !nonzero(v.y);
        }
        for (int k = tid; k < NC; k += NT) {
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T f = s_fro[m][k].x;
                q = q && (!nonzero(f) || f == one);
            }
            q = q && !nonzero(s_PM[k].x) && !is_nan(s_Io[k]);
            if (STR) {
                const T2 a = s_so01[k];
                q = q && !nonzero(a.x) && !nonzero(a.y) && !nonzero(s_so2d[k].x);
            }
        }
        quiet = __syncthreads_and(q);
    }
    if (quiet) {
        for (int k = tid; k < TW * TH; k += NT) {
            const int lx = H + k % TW, ly = H + k / TW, i = x0 + lx, j = y0 + ly;
            if (i >= nr || j >= nz) continue;
            const int kc = ly * CW + lx, c = j * nr + i;
            T phi = zero, M = zero;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T2 fr = s_fro[m][kc];
                const bool here = pos(fr.x);
                if (here) { phi += fr.x; M += fr.x * fr.y; }
                O.fr[m][c] = here ? fr : V::mk(zero, zero);
            }
            O.I[c] = pos(M) ? s_Io[kc] : 0.0;
            if (STR) {
                O.s01[c] = V::mk(zero, zero);
                O.s2d[c] = V::mk(zero, pos(phi) && pos(M) ? s_so2d[kc].y : zero);
            }
            const T2 ec = s_PM[kc];
            O.eosc[c] = ec;
            if (pos(phi)) {
                const T over = (NM == 1 ? ec.x : ec.x * (one / phi)) - p.p0[j];
                if (over > p.pmax[c]) p.pmax[c] = over;
                T speed = t_sqrt<T>(zero) + t_sqrt<T>(ec.y);
                if (!UNI) speed = speed * GE::ilen(P, i, j);
                if (is_nan(speed)) atomicOr(&p.scal->status, 2);
                speed_max = max_nonneg(speed_max, speed);
            }
        }
        for (int k = tid; k < (TW + 1) * (TH + 1); k += NT) {
            const int i = ox + k % (TW + 1), j = oy + k / (TW + 1);
            if (i > nr || j > nz) continue;
            if ((i < ox + TW || last_x) && (j < oy + TH || last_y)) O.v[j * nv + i] = V::mk(zero, zero);
        }
    } else {

    // ---- phase 0: artificial viscosity and total pressure from the equation of state of
    // the current state, which the previous step (or the Courant-rate pass) left in the
    // cache: (p_m, c^2) for one material, (p_hat, max c_m^2) for several; peak over-pressure
    // (owner)
    for (int k = tid; k < NC; k += NT) {
        const int lx = k % CW, ly = k / CW, i = x0 + lx, j = y0 + ly;
        if (i < 0 || i >= nr || j < 0 || j >= nz) {
            s_PM[k] = V::mk(zero, zero);
            if (PBPHI) s_pbphi[k] = V::mk(zero, zero);
            continue;
        }
        const T2 ec = s_PM[k];
        T phat = zero, phi = zero, mass = zero, r1 = zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T2 fr = s_fro[m][k];
            if (pos(fr.x)) {
                if (NM == 1) phat += fr.x * ec.x;
                phi += fr.x;
                mass += fr.x * fr.y;
                r1 = fr.y;
            }
        }
        if (NM > 1) phat = ec.x;
        const T c2m = ec.y, p1 = ec.x;
        T Pc = zero, pbar = zero;
        if (pos(phi)) {
            const T2 va = s_vo[ly * VW + lx], vb = s_vo[ly * VW + lx + 1];
            const T2 vc = s_vo[(ly + 1) * VW + lx + 1], vd = s_vo[(ly + 1) * VW + lx];
            const T uL = half * (va.x + vd.x), uR = half * (vb.x + vc.x);
            const T uB = half * (va.y + vb.y), uT = half * (vd.y + vc.y);
            const T div = (GE::flux_r(P, i, j, uL, uR) + p.A_Z[i] * (uT - uB)) * GE::ivol(P, i, j);
            const T cs = t_sqrt<T>(c2m);
            const T iphi = NM == 1 ? one : one / phi;
            pbar = NM == 1 ? p1 : phat * iphi;
            T q = zero;
            if (neg(div)) {
                const T rb = NM == 1 ? r1 : mass * iphi;
                const T Lc = GE::len(P, i, j);
                q = rb * (P.cq * (UNI ? P.dx2 : Lc * Lc) * div * div - P.cl * Lc * cs * div);
            }
            Pc = phat + phi * q;
            if (i >= ox && i < ox + TW && j >= oy && j < oy + TH) {
                const int c = j * nr + i;
                const T over = pbar - p.p0[j];
                if (over > p.pmax[c]) p.pmax[c] = over;
            }
        }
        s_PM[k] = V::mk(Pc, mass * GE::vol(P, i, j));
        if (PBPHI) s_pbphi[k] = V::mk(pbar, phi);
    }
    __syncthreads();

    // ---- phase 1: corner forces, gravity, PML psi1, Lagrangian velocity, BCs
    constexpr int R1 = CW - 1;
    for (int k = tid; k < R1 * (CH - 1); k += NT) {
        const int lx = 1 + k % R1, ly = 1 + k / R1, i = x0 + lx, j = y0 + ly;
        const int kv = ly * VW + lx;
        if (i < 0 || i > nr || j < 0 || j > nz) {
            s_vL[kv] = V::mk(zero, zero);
            s_mv[kv] = zero;
            s_dK[kv] = zero;
            continue;
        }
        const bool own = i >= ox && (i < ox + TW || (last_x && i <= nr)) && j >= oy && (j < oy + TH || (last_y && j <= nz));
        const int v = j * nv + i;
        T Pc[4] = {zero, zero, zero, zero}, Pp[4] = {zero, zero, zero, zero};
        T devr_rad = zero, devz_rad = zero, devr_ver = zero, devz_ver = zero, mass = zero;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ci = (q == 0 || q == 3) ? i - 1 : i;
            const int cj = (q < 2) ? j - 1 : j;
            if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
            const int kc = (cj - y0) * CW + (ci - x0);
            const T2 pm = s_PM[kc];
            Pc[q] = pm.x;
            mass += T(0.25) * pm.y;
            if (STR || P.pr > 0 || P.pb > 0) {
                T phi;
                if (PBPHI) {
                    phi = s_pbphi[kc].y;
                } else {
                    const T f = s_fro[0][kc].x;
                    phi = pos(f) ? f : zero;
                }
                Pp[q] = pm.x - phi * p.p0[cj];
                if (STR) {
                    const T2 s01 = s_so01[kc];
                    const T srz = s_so2d[kc].x;
                    const T Srr = phi * s01.x, Szz = phi * s01.y, Srz = phi * srz;
                    const T Stt = -(Srr + Szz);
                    const T hr = GE::half_v_dr(P, ci, cj), hz = half * p.A_Z[ci];
                    const T hoop = GE::quarter_v_rc(P, ci, cj);
                    const T sr = (q == 2 || q == 1) ? one : -one;
                    const T sz = (q == 2 || q == 3) ? one : -one;
                    devr_rad += sr * hr * Srr - hoop * Stt;
                    devz_rad += sr * hr * Srz;
                    devr_ver += sz * hz * Srz;
                    devz_ver += sz * hz * Szz;
                }
            }
        }
        const T ARb = UNI ? p.A_R[i] : (j > 0 ? GE::area_r(P, i, j - 1) : zero);
        const T ARt = UNI ? ARb : (j < nz ? GE::area_r(P, i, j) : zero);
        const T AZl = i > 0 ? p.A_Z[i - 1] : zero, AZr = i < nr ? p.A_Z[i] : zero;
        const T Fr = (UNI ? half * ARb * (((Pc[0] + Pc[3]) - Pc[1]) - Pc[2])
                          : half * (ARb * (Pc[0] - Pc[1]) + ARt * (Pc[3] - Pc[2]))) + (devr_rad + devr_ver);
        const T Fz = half * (AZl * (Pc[0] - Pc[3]) + AZr * (Pc[1] - Pc[2])) + (devz_rad + devz_ver);
        T psr = zero, psz = zero;
        if (j < P.pb) {
            const T d = p.dB_v[j];
            T4 a = p.pb_v[v];
            const T Tr = (UNI ? half * ARb * (((Pp[0] + Pp[3]) - Pp[1]) - Pp[2])
                              : half * (ARb * (Pp[0] - Pp[1]) + ARt * (Pp[3] - Pp[2]))) + devr_rad;
            const T rl = one - P.alpha_b * dt;
            a.z = a.z * rl - dt * d * Tr;
            a.w = a.w * rl - dt * d * devz_rad;
            if (own) store_pair(&O.pb_v[v], 1, V::mk(a.z, a.w));
            psr += a.z; psz += a.w;
        }
        if (i > nr - P.pr) {
            const int kk = j * P.pr + (i - (nr - P.pr + 1));
            const T d = strip_row_v(p, j, nz) ? p.dR_v[i] : zero;
            T4 a = p.pr_v[kk];
            const T Tz = half * (AZl * (Pp[0] - Pp[3]) + AZr * (Pp[1] - Pp[2])) + devz_ver;
            const T rl = one - P.alpha_r * dt;
            a.z = a.z * rl - dt * d * devr_ver;
            a.w = a.w * rl - dt * d * Tz;
            if (own) store_pair(&O.pr_v[kk], 1, V::mk(a.z, a.w));
            psr += a.z; psz += a.w;
        }
        const T2 vo = s_vo[kv];
        T vr = zero, vz = zero;
        if (pos(mass)) {
            // no net force and no gravity: v^L = v (the same value the update would give,
            // up to the sign of a zero) without the reciprocal
            const T fr_ = Fr - psr, fz_ = Fz - psz;
            const bool acc = nonzero(fr_) || nonzero(fz_) || nonzero(P.g);
            if (warp_any(acc) && acc) {
                const T im = one / mass;
                vr = vo.x + dt * (fr_ * im);
                vz = vo.y + dt * (fz_ * im - P.g);
            } else {
                vr = vo.x;
                vz = vo.y;
            }
        }
        if (i == 0 || i == nr) vr = zero;
        if (j == 0) {
            vz = zero;
            if (P.bc_bottom == SALEC_BOTTOM_NOSLIP) vr = zero;
        }
        if (j == nz && P.bc_top == SALEC_TOP_WALL) vz = zero;
        s_vL[kv] = V::mk(vr, vz);
        s_mv[kv] = mass;
        const T dvr = vr - vo.x, dvz = vz - vo.y;
        s_dK[kv] = half * mass * (dvr * dvr + dvz * dvz);
    }
    __syncthreads();

    // ---- phase 2: Lagrangian cell update from v^L
    constexpr int R2 = CW - 2;
    for (int k = tid; k < R2 * (CH - 2); k += NT) {
        const int lx = 1 + k % R2, ly = 1 + k / R2, i = x0 + lx, j = y0 + ly;
        const int kc = ly * CW + lx;
        if (i < 0 || i >= nr || j < 0 || j >= nz) continue;
        const int c = j * nr + i;
        const bool own = i >= ox && i < ox + TW && j >= oy && j < oy + TH;
        T phi;
        if (PBPHI) {
            phi = s_pbphi[kc].y;
        } else {
            const T f = s_fro[0][kc].x;
            phi = pos(f) ? f : zero;
        }
        if (!pos(phi)) {
#pragma unroll
            for (int m = 0; m < NM; ++m) s_frL[m][kc] = V::mk(zero, zero);
            s_VL[kc] = GE::vol(P, i, j);
            s_IL[kc] = 0.0;
            if (STR) { s_sL01[kc] = V::mk(zero, zero); s_sL2d[kc] = V::mk(zero, zero); }
            // an empty cell's psi2 is carried over unchanged
            if (own && j < P.pb) O.pb_psi2[c] = p.pb_psi2[c];
            if (own && i >= nr - P.pr) {
                const int kk = j * P.pr + (i - (nr - P.pr));
                O.pr_psi2[kk] = p.pr_psi2[kk];
            }
            continue;
        }
        const T2 va = s_vL[ly * VW + lx], vb = s_vL[ly * VW + lx + 1];
        const T2 vc = s_vL[(ly + 1) * VW + lx + 1], vd = s_vL[(ly + 1) * VW + lx];
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
        const T2 pm = s_PM[kc];
        const T Pc = pm.x, M = pm.y;
        T work = zero, Pi_rad = -Pc * rad_flux, Pi_ver = -Pc * ver_flux;
        T dvr_dz = zero, dvz_dr = zero, srr = zero, szz = zero, srz = zero, D = zero;
        if (STR) {
            const T2 s01 = s_so01[kc], s2d = s_so2d[kc];
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
            if (own) O.pb_psi2[c] = a;
            psi2 += a;
        }
        if (i >= nr - P.pr) {
            const int kk = j * P.pr + (i - (nr - P.pr));
            T a = p.pr_psi2[kk];
            a = a * (one - P.alpha_r * dt) - dt * (strip_row_c(p, j) ? p.dR_c[i] : zero) * Pi_ver;
            if (own) O.pr_psi2[kk] = a;
            psi2 += a;
        }
        const T dE = -Pc * dV + work - dt * psi2;
        const double Ic = s_Io[kc];
        const bool add_dE = pos(M) && nonzero(dE);
        double ILnew = Ic;
        if (warp_any(add_dE) && add_dE) ILnew = Ic + double(dE / M);
        s_IL[kc] = ILnew;
        s_VL[kc] = VLc;
        const T dVmat = phi * dV;
        bool bad = false;
        T G = zero, Y = zero, iepsf = zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T2 fr = s_fro[m][kc];
            if (pos(fr.x)) {
                const T Vm = fr.x * Vc;
                const T VmL = NM == 1 ? Vm + dVmat : Vm + fr.x / phi * dVmat;
                bad |= !pos(VmL) || !pos(fr.y);     // non-positive Lagrangian volume or density
                // unchanged volume: V_m / V_m^L is exactly 1 (no division)
                s_frL[m][kc] = V::mk(VmL / VLc, warp_any(nonzero(dV)) ? fr.y * (Vm / VmL) : fr.y);
                if (STR && P.mat[m].strength == SALEC_STRENGTH_COLLINS) {
                    const MatT<T>& mm = P.mat[m];
                    const T pb = s_pbphi[kc].x;
                    G += fr.x * mm.G;
                    Y += fr.x * yield_eval<T>(mm, pb, D, T(Ic), fr.y);
                    T ef = mm.B_dam * (pb - mm.p_bd);
                    ef = ef < mm.eps_fb ? mm.eps_fb : ef;
                    iepsf += fr.x / ef;
                }
            } else {
                s_frL[m][kc] = V::mk(zero, zero);
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
                    const T kq = Y / sq;
                    nrr *= kq; nzz *= kq; nrz *= kq;
                    D += (sq - Y) / (T(1.7320508075688772) * G) * iepsf;
                    D = D > one ? one : D;
                }
                srr = nrr; szz = nzz; srz = nrz;
            } else {
                srr = zero; szz = zero; srz = zero;
            }
            s_sL01[kc] = V::mk(srr, szz);
            s_sL2d[kc] = V::mk(srz, D);
        }
    }
    __syncthreads();

    // ---- phase 3a: donor-cell remap of the cells; face mass fluxes into shared memory
    {
        TileDonor<T, NM, STR> dn;
#pragma unroll
        for (int m = 0; m < NM; ++m) dn.frL[m] = s_frL[m];
        dn.IL = s_IL;
        dn.sL01 = s_sL01;
        dn.sL2d = s_sL2d;
        constexpr int R3 = CW - 4;
        for (int k = tid; k < R3 * (CH - 4); k += NT) {
            const int lx = 2 + k % R3, ly = 2 + k / R3, i = x0 + lx, j = y0 + ly;
            if (i < 0 || i >= nr || j < 0 || j >= nz) continue;
            const int kc = ly * CW + lx, c = j * nr + i;
            const bool own = i >= ox && i < ox + TW && j >= oy && j < oy + TH;
            Acc<T, NM> acc;
            const T VLc = s_VL[kc];
            const double ILc = s_IL[kc];
#pragma unroll
            for (int m = 0; m < NM; ++m) { acc.Vm[m] = zero; acc.Mm[m] = zero; }
            acc.dI = zero;
            acc.S[0] = acc.S[1] = acc.S[2] = acc.S[3] = zero;
            const bool strip = j < P.pb || i >= nr - P.pr;
            T FRm = zero, FRe = zero, FZm = zero, FZe = zero;
            T fm, fe;
            // left face r_i: positive dV flows from (i-1,j) into this cell
            {
                T dV = zero;
                if (i != 0 && i != nr) {
                    const T u = T(0.5) * (s_vL[ly * VW + lx].x + s_vL[(ly + 1) * VW + lx].x);
                    dV = dt * GE::area_r(P, i, j) * u;
                }
                T sm = zero;
                if (!warp_any(nonzero(dV))) {
                } else if (pos(dV)) { move_s<T, NM, STR>(dn, kc - 1, dV, one, ILc, strip, acc, fm, fe); sm = fm; FRm -= fm; FRe -= fe; }
                else if (neg(dV)) { move_s<T, NM, STR>(dn, kc, -dV, -one, ILc, strip, acc, fm, fe); sm = -fm; FRm += fm; FRe += fe; }
                s_dMR[ly * VW + lx] = sm;
            }
            // right face r_{i+1}
            {
                T dV = zero;
                if (i + 1 != nr) {
                    const T u = T(0.5) * (s_vL[ly * VW + lx + 1].x + s_vL[(ly + 1) * VW + lx + 1].x);
                    dV = dt * GE::area_r(P, i + 1, j) * u;
                }
                T sm = zero;
                if (!warp_any(nonzero(dV))) {
                } else if (pos(dV)) { move_s<T, NM, STR>(dn, kc, dV, -one, ILc, strip, acc, fm, fe); FRm += fm; FRe += fe; sm = fm; }
                else if (neg(dV)) { move_s<T, NM, STR>(dn, kc + 1, -dV, one, ILc, strip, acc, fm, fe); FRm -= fm; FRe -= fe; sm = -fm; }
                // the region's last column also records its right faces (the vertex remap
                // reads them); the grid's right wall carries nothing
                if (i == nr - 1) s_dMR[ly * VW + lx + 1] = zero;
                else if (lx == CW - 3) s_dMR[ly * VW + lx + 1] = sm;
            }
            // bottom face z_j
            {
                T dV = zero;
                if (j != 0 && !(j == nz && P.bc_top == SALEC_TOP_WALL)) {
                    const T u = T(0.5) * (s_vL[ly * VW + lx].y + s_vL[ly * VW + lx + 1].y);
                    dV = dt * p.A_Z[i] * u;
                }
                T sm = zero;
                if (!warp_any(nonzero(dV))) {
                } else if (pos(dV)) { move_s<T, NM, STR>(dn, kc - CW, dV, one, ILc, strip, acc, fm, fe); sm = fm; FZm -= fm; FZe -= fe; }
                else if (neg(dV)) { move_s<T, NM, STR>(dn, kc, -dV, -one, ILc, strip, acc, fm, fe); sm = -fm; FZm += fm; FZe += fe; }
                s_dMZ[ly * CW + lx] = sm;
            }
            // top face z_{j+1}: above the domain only outflow (inflow is void)
            {
                T dV = zero;
                if (!(j + 1 == nz && P.bc_top == SALEC_TOP_WALL)) {
                    const T u = T(0.5) * (s_vL[(ly + 1) * VW + lx].y + s_vL[(ly + 1) * VW + lx + 1].y);
                    dV = dt * p.A_Z[i] * u;
                }
                T sm = zero;
                if (!warp_any(nonzero(dV))) {
                } else if (pos(dV)) {
                    move_s<T, NM, STR>(dn, kc, dV, -one, ILc, strip, acc, fm, fe);
                    FZm += fm; FZe += fe; sm = fm;
                    if (j == nz - 1 && own) t_out += double(fm);
                } else if (neg(dV) && j + 1 < nz) {
                    move_s<T, NM, STR>(dn, kc + CW, -dV, one, ILc, strip, acc, fm, fe); FZm -= fm; FZe -= fe; sm = -fm;
                }
                // the region's last row also records its top faces; the top of the grid
                // records the outflow
                if (j == nz - 1 || ly == CH - 3) s_dMZ[(ly + 1) * CW + lx] = sm;
            }
            // new state in increment form (as the phase kernels)
            const T Vc = GE::vol(P, i, j);
            T Vm[NM], Mm[NM], rn[NM];
            T MLtot = zero, VLmat = zero, dMtot = zero, dVtot = zero;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T2 fl = s_frL[m][kc];
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
                const T2 a = s_sL01[kc], b = s_sL2d[kc];
                s0 = a.x + (acc.S[0] - a.x * dVtot) * iv;
                s1 = a.y + (acc.S[1] - a.y * dVtot) * iv;
                s2 = b.x + (acc.S[2] - b.x * dVtot) * iv;
                Dm = b.y + (acc.S[3] - b.y * dVtot) * iv;
            }
            T Mkeep = zero, Vkeep = zero, fnew[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                fnew[m] = Vm[m] / Vc;
                if (fnew[m] < P.f_min) {
                    const bool tally = own && nonzero(Mm[m]);
                    if (warp_any(tally) && tally) t_disc += double(Mm[m]);
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
                    T2 a = p.pb_c[c];
                    const T rl = one - P.alpha_b * dt;
                    a.x = a.x * rl + d * FRm;
                    a.y = a.y * rl + d * FRe;
                    if (own) O.pb_c[c] = a;
                    dsum += d; phi1 += a.x; phi3 += a.y;
                }
                if (inR) {
                    const int kk = j * P.pr + (i - (nr - P.pr));
                    const T d = strip_row_c(p, j) ? p.dR_c[i] : zero;
                    T2 a = p.pr_c[kk];
                    const T rl = one - P.alpha_r * dt;
                    a.x = a.x * rl + d * FZm;
                    a.y = a.y * rl + d * FZe;
                    if (own) O.pr_c[kk] = a;
                    dsum += d; phi1 += a.x; phi3 += a.y;
                }
                if (pos(Mkeep) && pos(dsum)) {
                    const T Mref = Vkeep * p.rho_ref[j];
                    const T dM = -dt * (dsum * (Mkeep - Mref) + phi1);
                    const double dEp = -double(dt) * (double(dsum) * (double(Mkeep) * Ic - double(Mref) * p.I_ref[j]) + double(phi3));
                    const T Mnew = Mkeep + dM;
                    if (!pos(Mnew)) atomicOr(&p.scal->status, 1);
                    if (own) t_pml += double(dM);
                    kappa = one + dM / Mkeep;
                    Ic = Ic + (dEp - Ic * double(dM)) / double(Mnew);
                }
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T2 f = pos(Vm[m]) ? V::mk(fnew[m], kappa * rn[m]) : V::mk(zero, zero);
                s_frn[m][kc] = f;
                if (own) O.fr[m][c] = f;
            }
            s_In[kc] = Ic;
            if (is_nan(Ic)) atomicOr(&p.scal->status, 2);
            if (STR && own) {
                O.s01[c] = V::mk(s0, s1);
                O.s2d[c] = V::mk(s2, Dm);
                s_Dn[kc] = Dm;
            }
        }
    }
    __syncthreads();

    // ---- phase 3b: momentum remap on the dual grid, PML phi2, heat per vertex
    {
        // face mass fluxes from shared memory; faces outside the grid carry nothing
        auto dMR_s = [&](int fx, int fy, int jj) -> T { return (jj < 0 || jj >= nz) ? zero : s_dMR[fy * VW + fx]; };
        auto dMZ_s = [&](int fx, int fy, int ii) -> T { return (ii < 0 || ii >= nr) ? zero : s_dMZ[fy * CW + fx]; };
        // dual mass flux between vertices (lx,ly) and (lx+1,ly), grid (i,j)
        auto dual_R_s = [&](int lx, int ly, int j) -> T {
            return T(0.25) * (dMR_s(lx, ly - 1, j - 1) + dMR_s(lx + 1, ly - 1, j - 1) + dMR_s(lx, ly, j) + dMR_s(lx + 1, ly, j));
        };
        // between (lx,ly) and (lx,ly+1); j == nz: out through the top
        auto dual_Z_s = [&](int lx, int ly, int i, int j) -> T {
            if (j == nz) return T(0.5) * (dMZ_s(lx - 1, ly, i - 1) + dMZ_s(lx, ly, i));
            return T(0.25) * (dMZ_s(lx - 1, ly, i - 1) + dMZ_s(lx - 1, ly + 1, i - 1) + dMZ_s(lx, ly, i) + dMZ_s(lx, ly + 1, i));
        };
        constexpr int RB = TW + 1;
        for (int k = tid; k < RB * (TH + 1); k += NT) {
            const int lx = H + k % RB, ly = H + k / RB, i = x0 + lx, j = y0 + ly;
            if (i > nr || j > nz) continue;
            const int kv = ly * VW + lx, v = j * nv + i;
            const bool own = (i < ox + TW || last_x) && (j < oy + TH || last_y);
            const T2 vL = s_vL[kv];
            DualFace<T> oR = {zero, zero, zero, zero}, oZ = {zero, zero, zero, zero};
            DualFace<T> iR = {zero, zero, zero, zero}, iZ = {zero, zero, zero, zero};
            if (i < nr) {
                const T f = dual_R_s(lx, ly, j);
                oR = dual_face<T>(f, pos(f) ? vL : s_vL[kv + 1]);
            }
            {
                const T f = dual_Z_s(lx, ly, i, j);
                oZ = dual_face<T>(f, (pos(f) || j == nz) ? vL : s_vL[kv + VW]);
            }
            if (i > 0) {
                const T f = dual_R_s(lx - 1, ly, j);
                iR = dual_face<T>(f, pos(f) ? s_vL[kv - 1] : vL);
            }
            if (j > 0) {
                const T f = dual_Z_s(lx, ly - 1, i, j - 1);
                iZ = dual_face<T>(f, pos(f) ? s_vL[kv - VW] : vL);
            }
            const T m0 = s_mv[kv];
            T m = m0, pr = m0 * vL.x, pz = m0 * vL.y;
            T kin = half * m0 * (vL.x * vL.x + vL.y * vL.y);
            m += iR.f; kin += iR.e;
            m -= oR.f; kin -= oR.e;
            m += iZ.f; kin += iZ.e;
            m -= oZ.f; kin -= oZ.e;
            const T inRr = iR.fr, inRz = iR.fz, outRr = oR.fr, outRz = oR.fz;
            const T inZr = iZ.fr, inZz = iZ.fz, outZr = oZ.fr, outZz = oZ.fz;
            const bool top = own && j == nz;
            if (warp_any(top) && top) t_zmom += double(outZz);
            pr += (inRr - outRr) + (inZr - outZr);
            pz += (inRz - outRz) + (inZz - outZz);
            const T dKv = s_dK[kv];
            const bool quiet = !nonzero(pr) && !nonzero(pz) && !nonzero(kin) && !nonzero(dKv);
            T kheat = zero, im = zero;
            bool have_im = false;
            if (pos(m) && warp_any(!quiet) && !quiet) {
                im = one / m;
                have_im = true;
                const T dKr = kin - half * (pr * pr + pz * pz) * im;
                kheat = (dKv + dKr) * im;
            }
            s_kheat[kv] = kheat;
            T dsum = zero, a2r = zero, a2z = zero;
            if (j < P.pb) {
                const T d = p.dB_v[j];
                T4 a = p.pb_v[v];
                const T rl = one - P.alpha_b * dt;
                a.x = a.x * rl + d * (outRr - inRr);
                a.y = a.y * rl + d * (outRz - inRz);
                if (own) store_pair(&O.pb_v[v], 0, V::mk(a.x, a.y));
                dsum += d; a2r += a.x; a2z += a.y;
            }
            if (i > nr - P.pr) {
                const int kk = j * P.pr + (i - (nr - P.pr + 1));
                const T d = strip_row_v(p, j, nz) ? p.dR_v[i] : zero;
                T4 a = p.pr_v[kk];
                const T rl = one - P.alpha_r * dt;
                a.x = a.x * rl + d * (outZr - inZr);
                a.y = a.y * rl + d * (outZz - inZz);
                if (own) store_pair(&O.pr_v[kk], 0, V::mk(a.x, a.y));
                dsum += d; a2r += a.x; a2z += a.y;
            }
            if (j < P.pb || i > nr - P.pr) {
                pr = pr - dt * (dsum * pr + a2r);
                pz = pz - dt * (dsum * pz + a2z);
            }
            T vr = zero, vz = zero;
            const bool moving = nonzero(pr) || nonzero(pz);
            if (pos(m) && warp_any(moving) && moving) {
                // no material in any adjacent cell after the clean-up: no momentum
                bool occupied = false;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ci = (q == 0 || q == 3) ? i - 1 : i;
                    const int cj = (q < 2) ? j - 1 : j;
                    if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                    const int kc = (cj - y0) * CW + (ci - x0);
#pragma unroll
                    for (int mm = 0; mm < NM; ++mm) occupied |= pos(s_frn[mm][kc].x);
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
            const T2 vnew = V::mk(vr, vz);
            s_vn[kv] = vnew;
            if (own) O.v[v] = vnew;
        }
    }
    __syncthreads();

    // ---- phase 3c: heat to the own cells; the Courant rate of the new state (Eq. 14)
    for (int k = tid; k < TW * TH; k += NT) {
        const int lx = H + k % TW, ly = H + k / TW, i = x0 + lx, j = y0 + ly;
        if (i >= nr || j >= nz) continue;
        const int kc = ly * CW + lx, c = j * nr + i;
        T M = zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T2 fr = s_frn[m][kc];
            M += fr.x * fr.y;
        }
        double Ic = s_In[kc];
        const int ka = ly * VW + lx;
        if (pos(M)) {
            const T add = T(0.25) * (s_kheat[ka] + s_kheat[ka + 1] + s_kheat[ka + VW + 1] + s_kheat[ka + VW]);
            if (warp_any(nonzero(add)) && nonzero(add)) Ic += double(add);
        }
        O.I[c] = Ic;
        // the equation of state of the new state, as phase 0 of the next step would form it
        // (into the cache it reads), and the rate (|v| + c) / L for the next step's dt.  A
        // cell whose fractions, densities, energy and damage are bitwise those of the
        // current state keeps its cached values (same inputs, same results).
        T phi = zero;
        T2 ec;
        const T D = STR ? s_Dn[kc] : zero;
        bool same = __double_as_longlong(Ic) == __double_as_longlong(p.I[c]);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T2 fn = s_frn[m][kc], fo = p.fr[m][c];
            same = same && fn.x == fo.x && fn.y == fo.y;
            if (pos(fn.x)) phi += fn.x;
        }
        if (STR) same = same && D == p.s2d[c].y;
        if (!warp_any(!same)) {
            ec = p.eosc[c];
        } else {
            T c2m = zero, phat = zero, p1 = zero;
            const T In = T(Ic);
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T2 fr = s_frn[m][kc];
                if (pos(fr.x)) {
                    T pm, c2;
                    eos_eval<T>(P.mat[m], fr.y, In, pm, c2);
                    const T pmin = (one - D) * P.mat[m].p_t * expansion_weight(P.mat[m], fr.y);
                    pm = pm < pmin ? pmin : pm;
                    phat += fr.x * pm;
                    c2m = max_nonneg(c2m, c2);
                    p1 = pm;
                }
            }
            ec = V::mk(NM == 1 ? p1 : phat, c2m);
        }
        O.eosc[c] = ec;
        const T c2m = ec.y;
        if (pos(phi)) {
            const T2 va = s_vn[ka], vb = s_vn[ka + 1], vc = s_vn[ka + VW + 1], vd = s_vn[ka + VW];
            T w = va.x * va.x + va.y * va.y;
            w = max_nonneg(w, vb.x * vb.x + vb.y * vb.y);
            w = max_nonneg(w, vc.x * vc.x + vc.y * vc.y);
            w = max_nonneg(w, vd.x * vd.x + vd.y * vd.y);
            T speed = t_sqrt<T>(w) + t_sqrt<T>(c2m);
            if (!UNI) speed = speed * GE::ilen(P, i, j);
            if (is_nan(speed)) atomicOr(&p.scal->status, 2);
            speed_max = max_nonneg(speed_max, speed);
        }
    }

    }   // not quiescent
    if (tid == 0) O.rest_out[tile] = quiet ? 1 : 0;
    }   // tiles

    // ---- reductions.  The tallies (FP64) are rare (top row, strips, clean-up): a warp that
    // holds one sums it and adds it with one atomic per tally, so no other warp issues FP64
    // work for them.  The Courant maximum of every block goes through warp 0.
    {
        const int lane = tid & 31, w = tid >> 5;
        const bool any_tally = nonzero(t_out) || nonzero(t_disc) || nonzero(t_pml) || nonzero(t_zmom);
        if (__any_sync(0xffffffffu, any_tally)) {
            double sv[4] = {t_out, t_disc, t_pml, t_zmom};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q) sv[q] += __shfl_down_sync(0xffffffffu, sv[q], o);
            if (lane == 0) {
                DevScalars* s = p.scal;
                if (sv[0] != 0.0) atomicAdd(&s->mass_out, sv[0]);
                if (sv[1] != 0.0) atomicAdd(&s->mass_discarded, sv[1]);
                if (sv[2] != 0.0) atomicAdd(&s->mass_pml, sv[2]);
                if (sv[3] != 0.0) atomicAdd(&s->zmom_out, sv[3]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) speed_max = max_nonneg(speed_max, __shfl_down_sync(0xffffffffu, speed_max, o));
        unsigned long long* s_bits = reinterpret_cast<unsigned long long*>(s_red);
        if (lane == 0) s_bits[w] = (unsigned long long)__double_as_longlong(double(speed_max));
        __syncthreads();
        if (w == 0) {
            unsigned long long b = lane < NT / 32 ? s_bits[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
            if (lane == 0) {
                DevScalars* s = p.scal;
                atomicMax(&s->maxbits, b);
                if (blockIdx.x == 0) {
                    s->t += s->dt;
                    s->dt_prev = s->dt;
                    s->nstep += 1ull;
                }
            }
        }
    }
}

// ---- tiles at rest.  A tile that the step before took through the quiescent path, and
// whose eight neighbours it took through it too, has an unchanged frame that still passes
// every test of that path; and its fields already are what that path writes (an absent
// material as zeros, no deviatoric stress, vertices at rest, an empty cell's energy zero).
// So its outputs are its inputs bit for bit, its peak over-pressure stays (the same
// pressure against the same reference as in the step before), and its Courant rate is
// that of its fastest sound speed: one square root of the largest c^2 of its cells on a
// uniform grid (the rounded square root is monotonic).  This kernel copies those tiles,
// one warp per tile with the loads of several rows in flight, and queues every other tile
// for the tile kernel.
constexpr int kRestThreads = 256;

template <typename T, int NM, bool STR, bool UNI, int TW, int TH>
__global__ void __launch_bounds__(kRestThreads) k_rest_tiles(const ParamsT<T> P, const OutPtrsT<T> O)
{
    typedef VT<T> V;
    typedef typename V::T2 T2;
    typedef Geo<T, UNI> GE;
    static_assert(TW == 32, "one lane per column of a tile");
    constexpr int R = NM == 1 ? 4 : 2;            // rows whose loads are in flight together
    const PtrsT<T>& p = P.p;
    const T zero = T(0);
    const int nr = P.nr, nz = P.nz, nv = nr + 1;
    const int nbx = (nr + TW - 1) / TW, nby = (nz + TH - 1) / TH;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * (kRestThreads / 32) + w;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        O.work_next->count = 0;
        O.work_next->next = 0;
        O.work_next->back = 0;
        O.work_next->copy_next = 0;
    }
    T c2max = zero, speed_max = zero;
    bool bad = false;
    if (tile < nbx * nby) {
        const int bx = tile % nbx, by = tile / nbx;
        bool rest = true;
        if (lane < 9) {
            const int tx = bx + lane % 3 - 1, ty = by + lane / 3 - 1;
            if (tx >= 0 && tx < nbx && ty >= 0 && ty < nby) rest = O.rest_in[ty * nbx + tx] != 0;
        }
        rest = __all_sync(0xffffffffu, rest);
        if (!rest) {
            // each tile is queued once a step: one that took the whole cycle in the step
            // before at the front, one queued only for a neighbour (most of these take the
            // quiescent path again) at the back, so that the long cycles start first and
            // the short ones fill the end of the kernel
            if (lane == 0) {
                if (O.rest_in[tile] == 0) {
                    const int q = atomicAdd(&O.work->count, 1);
                    if (q < nbx * nby) O.list[q] = tile;
                } else {
                    const int q = atomicAdd(&O.work->back, 1);
                    if (q < nbx * nby) O.list[nbx * nby - 1 - q] = tile;
                }
            }
        } else {
            if (lane == 0) O.rest_out[tile] = 1;
            const int i = bx * TW + lane, jb = by * TH, je = min(jb + TH, nz);
            if (i < nr) {
                for (int j0 = jb; j0 < je; j0 += R) {
                    T2 fr[R][NM], ec[R], sd[R];
                    double Ic[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (j0 + r >= je) break;
                        const int c = (j0 + r) * nr + i;
#pragma unroll
                        for (int m = 0; m < NM; ++m) fr[r][m] = p.fr[m][c];
                        Ic[r] = p.I[c];
                        ec[r] = p.eosc[c];
                        if (STR) sd[r] = p.s2d[c];
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (j0 + r >= je) break;
                        const int j = j0 + r, c = j * nr + i;
                        bool here = false;
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            O.fr[m][c] = fr[r][m];
                            here = here || pos(fr[r][m].x);
                        }
                        O.I[c] = Ic[r];
                        O.eosc[c] = ec[r];
                        if (STR) {
                            O.s01[c] = V::mk(zero, zero);
                            O.s2d[c] = sd[r];
                        }
                        if (here) {
                            const T c2 = ec[r].y;
                            if (!UNI || is_nan(c2) || neg(c2)) {
                                // the quiescent path's own arithmetic, cell by cell
                                T speed = t_sqrt<T>(zero) + t_sqrt<T>(c2);
                                if (!UNI) speed = speed * GE::ilen(P, i, j);
                                bad = bad || is_nan(speed);
                                speed_max = max_nonneg(speed_max, speed);
                            } else {
                                c2max = max_nonneg(c2max, c2);
                            }
                        }
                    }
                }
            }
            // the tile's vertices (with the grid's far edges on the last tiles) at rest
            const int jv = by == nby - 1 ? nz + 1 : jb + TH;
            const bool edge = lane == 0 && bx == nbx - 1 && bx * TW + TW == nr;
            for (int j = jb; j < jv; ++j) {
                if (i <= nr) O.v[j * nv + i] = V::mk(zero, zero);
                if (edge) O.v[j * nv + nr] = V::mk(zero, zero);
            }
        }
    }
    if (UNI) speed_max = max_nonneg(speed_max, t_sqrt<T>(zero) + t_sqrt<T>(c2max));
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&p.scal->status, 2);
    __shared__ unsigned long long sh[kRestThreads / 32];
    unsigned long long b = (unsigned long long)__double_as_longlong(double(speed_max));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    if (lane == 0) sh[w] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kRestThreads / 32; ++k) b = max(b, sh[k]);
        if (b != 0ull) atomicMax(&p.scal->maxbits, b);
    }
}

// ---- Tiles at rest copied beside the tile kernel (FP64 form) -----------------------------
// The rest-tile kernel above streams the tiles at rest before the tile kernel starts; the
// tile kernel then keeps the FP64 pipes busy with DRAM idle.  Here the two overlap: a scan
// kernel only queues the tiles (and flags the tiles at rest), and a copy kernel of one
// warp per SM, on a second stream, moves the tiles at rest with bulk tensor copies
// (global -> shared -> global, no registers in between) while the tile kernel computes on
// the same SMs.  Its CTA takes more than half of an SM's shared memory, so no SM holds two
// of them, and little enough that one fits beside a tile-kernel CTA.

constexpr int kCopyStages = 5;          // tiles whose loads a copy CTA keeps in flight

struct RestCopyArgs {
    int nr, nz;
    const unsigned char* rest_in;
    TileWork* work;         // copy_next: groups of 32 tiles handed out
    DevScalars* scal;
    double2* v;             // vertices of the copy written (the grid's last row and column)
};

// A tile is at rest when it and its eight neighbours (those inside the grid) took the
// quiescent path in the step that wrote the copy read here.
__device__ __forceinline__ bool tile_at_rest(const unsigned char* __restrict__ rest_in, int tile, int nbx, int nby)
{
    const int bx = tile % nbx, by = tile / nbx;
    int rest = 1;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int tx = bx + dx, ty = by + dy;
            if (tx >= 0 && tx < nbx && ty >= 0 && ty < nby) rest &= rest_in[ty * nbx + tx] != 0;
        }
    return rest != 0;
}

// One thread per tile: a tile at rest gets its flag for the next step (the copy kernel
// moves its fields); every other tile is queued for the tile kernel, as the rest-tile
// kernel queues it (front: took the whole cycle in the step before; back: queued for a
// neighbour).  Empties the next step's queue.
template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) k_rest_scan(const int nr, const int nz, const OutPtrsT<double> O)
{
    const int nbx = (nr + TW - 1) / TW, nby = (nz + TH - 1) / TH, ntiles = nbx * nby;
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile == 0) {
        O.work_next->count = 0;
        O.work_next->next = 0;
        O.work_next->back = 0;
        O.work_next->copy_next = 0;
    }
    if (tile >= ntiles) return;
    if (tile_at_rest(O.rest_in, tile, nbx, nby)) {
        O.rest_out[tile] = 1;
    } else if (O.rest_in[tile] == 0) {
        const int q = atomicAdd(&O.work->count, 1);
        if (q < ntiles) O.list[q] = tile;
    } else {
        const int q = atomicAdd(&O.work->back, 1);
        if (q < ntiles) O.list[ntiles - 1 - q] = tile;
    }
}

// The copy: one warp per CTA.  Lane 0 issues the bulk copies; the warp takes groups of 32
// tiles from a counter, tests them (one lane a tile) and copies those at rest through a
// ring of kCopyStages shared-memory stages: the (f, rho) of each material, the EoS cache
// and the energy of a tile in, the same out to the copy written, plus zeros for the
// tile's vertices.  Between the load and the store the warp forms the tile's Courant
// rates as the rest-tile kernel does (the largest c^2 of its cells with matter; NaN or
// negative c^2 cell by cell), for the running maximum that sets the next step's dt.
// Stage layout: (f, rho) of material m at m * FR, the EoS cache at NM * FR, I at
// (NM + 1) * FR.  The maps index: src/dst[m] (f, rho), [NM] I, [NM + 1] the EoS cache.
// A wait that runs out (2 s) sets status bit 8 and ends the copy.  32 registers a thread:
// the warp then fits into the quarter of the register file that the tile CTA's four warps
// in each SM sub-partition leave (4 x 120 x 32 of 16 384).
template <int NM, int TW, int TH>
__global__ void __maxnreg__(32) k_rest_copy(const __grid_constant__ RestCopy rc, const RestCopyArgs A)
{
    constexpr int FR = TW * TH * 16, FI = TW * TH * 8;
    constexpr int STAGE = (NM + 1) * FR + FI;
    constexpr int S = kCopyStages;
    extern __shared__ __align__(128) unsigned char copy_smem[];
    __shared__ __align__(8) uint64_t full[S];
    // the stages on a 128-byte boundary (the launch asks for 128 bytes more than they take)
    unsigned char* smem = copy_smem + ((128u - (tma::smem_u32(copy_smem) & 127u)) & 127u);
    unsigned char* zeros = smem + S * STAGE;          // TW x TH vertices of (0, 0)
    const int lane = threadIdx.x;
    const int nr = A.nr, nz = A.nz, nv = nr + 1;
    const int nbx = (nr + TW - 1) / TW, nby = (nz + TH - 1) / TH, ntiles = nbx * nby;
    const int ngroups = (ntiles + 31) / 32;
    for (int k = lane; k < TW * TH; k += 32) reinterpret_cast<double2*>(zeros)[k] = make_double2(0.0, 0.0);
    if (lane == 0) {
        for (int s = 0; s < S; ++s) tma::mbar_init(&full[s], 1);
        tma::fence_mbar_init();
    }
    tma::fence_async_smem();        // the zeros, for the tensor stores
    __syncwarp();

    // the warp's tiles at rest, in the order it takes them (warp-uniform)
    int grp = 0;
    unsigned mask = 0u;
    bool more = true;
    auto next_tile = [&]() -> int {
        while (mask == 0u && more) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&A.work->copy_next, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= ngroups) {
                more = false;
                break;
            }
            grp = g;
            const int t = g * 32 + lane;
            mask = __ballot_sync(0xffffffffu, t < ntiles && tile_at_rest(A.rest_in, t, nbx, nby));
        }
        if (mask == 0u) return -1;
        const int b = __ffs(mask) - 1;
        mask &= mask - 1u;
        return grp * 32 + b;
    };
    auto load = [&](int s, int tile) {     // lane 0
        unsigned char* st = smem + s * STAGE;
        const int x2 = 2 * TW * (tile % nbx), x1 = TW * (tile % nbx), y = TH * (tile / nbx);
        tma::mbar_expect_tx(&full[s], STAGE);
#pragma unroll
        for (int m = 0; m < NM; ++m) tma::load_2d(st + m * FR, &rc.src[m], x2, y, &full[s]);
        tma::load_2d(st + NM * FR, &rc.src[NM + 1], x2, y, &full[s]);
        tma::load_2d(st + (NM + 1) * FR, &rc.src[NM], x1, y, &full[s]);
    };

    int ring[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        ring[s] = next_tile();
        if (lane == 0 && ring[s] >= 0) load(s, ring[s]);
    }
    double c2max = 0.0, speed_max = 0.0;
    bool bad = false, failed = false;
    int n = 0;
    for (;; ++n) {
        const int s = n % S;
        const int tile = ring[s];
        if (tile < 0) break;
        if (!__all_sync(0xffffffffu, tma::mbar_wait(&full[s], (n / S) & 1))) {
            failed = true;
            break;
        }
        const unsigned char* st = smem + s * STAGE;
        const double2* ec = reinterpret_cast<const double2*>(st + NM * FR);
#pragma unroll 4
        for (int r = 0; r < TH; ++r) {
            const int k = r * TW + lane;
            bool here = false;
#pragma unroll
            for (int m = 0; m < NM; ++m) here = here || pos(reinterpret_cast<const double2*>(st + m * FR)[k].x);
            if (here) {
                const double c2 = ec[k].y;
                if (is_nan(c2) || neg(c2)) {
                    const double speed = t_sqrt<double>(0.0) + t_sqrt<double>(c2);
                    bad = bad || is_nan(speed);
                    speed_max = max_nonneg(speed_max, speed);
                } else {
                    c2max = max_nonneg(c2max, c2);
                }
            }
        }
        __syncwarp();
        const int bx = tile % nbx, by = tile / nbx;
        if (lane == 0) {
            const int x2 = 2 * TW * bx, x1 = TW * bx, y = TH * by;
#pragma unroll
            for (int m = 0; m < NM; ++m) tma::store_2d(&rc.dst[m], x2, y, st + m * FR);
            tma::store_2d(&rc.dst[NM + 1], x2, y, st + NM * FR);
            tma::store_2d(&rc.dst[NM], x1, y, st + (NM + 1) * FR);
            tma::store_2d(&rc.v, x2, y, zeros);
            tma::bulk_commit();
        }
        // the vertex box covers columns TW bx .. TW bx + TW - 1 and rows TH by .. TH by + TH - 1
        // (clipped to the grid); where the grid's last vertex row or column falls just
        // outside it, plain stores
        const int jb = TH * by, i = TW * bx + lane;
        if (by == nby - 1 && jb + TH == nz && i <= nr) A.v[nz * nv + i] = make_double2(0.0, 0.0);
        if (bx == nbx - 1 && TW * bx + TW == nr) {
            const int jv = by == nby - 1 ? nz + 1 : jb + TH;
            for (int j = jb + lane; j < jv; j += 32) A.v[j * nv + nr] = make_double2(0.0, 0.0);
        }
        // refill the stage of the tile before, once its stores have read it
        if (n > 0) {
            const int ps = (n - 1) % S;
            if (lane == 0) tma::bulk_wait_read<1>();
            __syncwarp();
            const int t2 = next_tile();
            ring[ps] = t2;
            if (lane == 0 && t2 >= 0) {
                tma::fence_async_smem();
                load(ps, t2);
            }
        }
    }
    if (lane == 0) {
        tma::bulk_wait_all();
        if (failed) {
            // the loads still in flight land before the CTA's shared memory is released
            const int pending = n == 0 ? S : S - 1;
            for (int d = 0; d < pending; ++d) {
                const int q = (n + d) % S;
                if (ring[q] >= 0) (void)tma::mbar_wait(&full[q], ((n + d) / S) & 1);
            }
            atomicOr(&A.scal->status, 8);
        }
    }
    speed_max = max_nonneg(speed_max, t_sqrt<double>(0.0) + t_sqrt<double>(c2max));
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&A.scal->status, 2);
    unsigned long long b = (unsigned long long)__double_as_longlong(speed_max);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    if (lane == 0 && b != 0ull) atomicMax(&A.scal->maxbits, b);
}

// The equation of state of the current state into the cache and its Courant rates into the
// running maximum (the first step of a sequence of fused steps, or after the host changed
// the state): the phase-0 arithmetic of both.  With rest (set to 1 for every tile before
// the launch) it also clears the rest flag of every tile that the quiescent path would not
// return bit for bit: one whose frame lies in a strip or under gravity, or one with a cell
// or vertex that fails the quiescence test, or whose fields differ from what that path
// writes (an absent material or an empty cell's energy not +0, deviatoric stress or a
// damage that the path zeroes, a peak over-pressure the path would raise).  A tile whose
// eight neighbours keep their flags too then has a quiescent frame and outputs equal to its
// inputs, so the first fused step copies it instead of queueing it.
template <typename T, int NM, bool STR, bool UNI, int TW, int TH>
__global__ void __launch_bounds__(kThreads) k_courant_rates(const ParamsT<T> P, unsigned char* __restrict__ rest)
{
    static_assert(TW == kBlockX && TH % kBlockY == 0, "a block of the pass lies in one tile");
    typedef VT<T> V;
    typedef typename V::T2 T2;
    typedef Geo<T, UNI> GE;
    const T zero = T(0);
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const PtrsT<T>& p = P.p;
    const int nr = P.nr;
    T speed = zero;
    bool q = true;          // cells outside the grid read as empty: quiescent
    if (i < nr && j < P.nz) {
        const int c = j * nr + i;
        T phi = zero, c2m = zero, phat = zero, p1 = zero;
        const T Ic = T(p.I[c]);
        const T D = STR ? p.s2d[c].y : zero;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T2 fr = p.fr[m][c];
            if (pos(fr.x)) {
                T pm, c2;
                eos_eval<T>(P.mat[m], fr.y, Ic, pm, c2);
                const T pmin = (T(1) - D) * P.mat[m].p_t * expansion_weight(P.mat[m], fr.y);
                pm = pm < pmin ? pmin : pm;
                phat += fr.x * pm;
                phi += fr.x;
                c2m = max_nonneg(c2m, c2);
                p1 = pm;
            }
        }
        const T ecx = NM == 1 ? p1 : phat;
        p.eosc[c] = V::mk(ecx, c2m);
        const int nv = nr + 1;
        const T2 va = p.v[j * nv + i], vb = p.v[j * nv + i + 1];
        const T2 vc = p.v[(j + 1) * nv + i + 1], vd = p.v[(j + 1) * nv + i];
        if (pos(phi)) {
            T w = va.x * va.x + va.y * va.y;
            w = max_nonneg(w, vb.x * vb.x + vb.y * vb.y);
            w = max_nonneg(w, vc.x * vc.x + vc.y * vc.y);
            w = max_nonneg(w, vd.x * vd.x + vd.y * vd.y);
            speed = t_sqrt<T>(w) + t_sqrt<T>(c2m);
            if (!UNI) speed = speed * GE::ilen(P, i, j);
            if (is_nan(speed)) atomicOr(&p.scal->status, 2);
        }
        if (rest) {
            // the quiescence test of the tile kernel on this cell and its corners, and its
            // outputs equal to its inputs
            q = !nonzero(va.x) && !nonzero(va.y) && !nonzero(vb.x) && !nonzero(vb.y) &&
                !nonzero(vc.x) && !nonzero(vc.y) && !nonzero(vd.x) && !nonzero(vd.y) &&
                !nonzero(ecx) && !is_nan(Ic);
            T M = zero;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const T2 fr = p.fr[m][c];
                if (pos(fr.x)) M += fr.x * fr.y;
                q = q && (fr.x == T(1) || (is_pzero(fr.x) && is_pzero(fr.y)));
            }
            if (!pos(M)) q = q && is_pzero(p.I[c]);
            if (STR) {
                const T2 a = p.s01[c], b = p.s2d[c];
                q = q && !nonzero(a.x) && !nonzero(a.y) && is_pzero(b.x) && ((pos(phi) && pos(M)) || is_pzero(b.y));
            }
            if (pos(phi)) {
                const T over = (NM == 1 ? ecx : ecx * (T(1) / phi)) - p.p0[j];
                q = q && !(over > p.pmax[c]);
            }
        }
    }
    if (rest) {
        // the frame of the tile: outside the strips, no gravity
        const int bx = blockIdx.x * kBlockX / TW, by = blockIdx.y * kBlockY / TH;
        const int x0 = bx * TW - 3, y0 = by * TH - 3;
        const bool frame = !nonzero(P.g) && y0 >= P.pb && x0 + TW + 6 <= nr - P.pr;
        if (!__syncthreads_and(q && frame) && threadIdx.x == 0 && threadIdx.y == 0)
            rest[by * ((nr + TW - 1) / TW) + bx] = 0;
    }
    __shared__ unsigned long long sh[kThreads / 32];
    const int tid = threadIdx.y * kBlockX + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) speed = max_nonneg(speed, __shfl_down_sync(0xffffffffu, speed, o));
    if ((tid & 31) == 0) sh[tid >> 5] = (unsigned long long)__double_as_longlong(double(speed));
    __syncthreads();
    if (tid != 0) return;
    unsigned long long b = sh[0];
    for (int w = 1; w < kThreads / 32; ++w) b = max(b, sh[w]);
    atomicMax(&p.scal->maxbits, b);
}

namespace {

template <typename T, int NM, bool STR, bool UNI>
struct Fused {
    typedef TileShape<T, NM, STR> S;
    typedef TileLayout<T, NM, STR, S::TW, S::TH> L;
    static_assert(S::TW == kFusedTileW && S::TH >= kFusedTileMinH, "tile count bound");
    static void* fn() { return reinterpret_cast<void*>(k_step_fused<T, NM, STR, UNI, S::TW, S::TH, S::NT, S::MINB>); }
    static int tiles(const ParamsT<T>& P) { return ((P.nr + S::TW - 1) / S::TW) * ((P.nz + S::TH - 1) / S::TH); }
    // the persistent grid: as many CTAs as the device holds at once
    static cudaError_t prepare(int* ctas)
    {
        auto k = k_step_fused<T, NM, STR, UNI, S::TW, S::TH, S::NT, S::MINB>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        int dev = 0, sms = 0, per_sm = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, S::NT, L::bytes);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) *ctas = sms * per_sm;
        return e;
    }
    static cudaError_t rest(const ParamsT<T>& P, const OutPtrsT<T>& O, cudaStream_t s)
    {
        constexpr int wpb = kRestThreads / 32;
        k_rest_tiles<T, NM, STR, UNI, S::TW, S::TH><<<(tiles(P) + wpb - 1) / wpb, kRestThreads, 0, s>>>(P, O);
        return cudaGetLastError();
    }
    static cudaError_t launch(const ParamsT<T>& P, const OutPtrsT<T>& O, cudaStream_t s)
    {
        k_step_fused<T, NM, STR, UNI, S::TW, S::TH, S::NT, S::MINB><<<O.ctas, S::NT, L::bytes, s>>>(P, O);
        return cudaGetLastError();
    }
    static cudaError_t rates(const ParamsT<T>& P, unsigned char* rest, cudaStream_t s)
    {
        const dim3 g((P.nr + kBlockX - 1) / kBlockX, (P.nz + kBlockY - 1) / kBlockY);
        k_courant_rates<T, NM, STR, UNI, S::TW, S::TH><<<g, dim3(kBlockX, kBlockY), 0, s>>>(P, rest);
        return cudaGetLastError();
    }
};

// dispatch on the material count, strength and grid form of a run
template <typename T, template <typename, int, bool, bool> class F, typename Fn>
cudaError_t dispatch(const ParamsT<T>& P, Fn&& fn)
{
    const bool st = P.any_strength != 0, un = P.uniform != 0;
#define SALEC_FUSED_CASE(NM_)                                                                        \
    case NM_:                                                                                         \
        if (un) return st ? fn(F<T, NM_, true, true>()) : fn(F<T, NM_, false, true>());               \
        return st ? fn(F<T, NM_, true, false>()) : fn(F<T, NM_, false, false>());
    switch (P.nmat) {
        SALEC_FUSED_CASE(1)
        SALEC_FUSED_CASE(2)
        SALEC_FUSED_CASE(3)
    default: return cudaErrorInvalidValue;
    }
#undef SALEC_FUSED_CASE
}

}  // namespace

template <typename T>
cudaError_t prepare_fused(const ParamsT<T>& P, int* ctas)
{
    return dispatch<T, Fused>(P, [&](auto f) { return decltype(f)::prepare(ctas); });
}

template <typename T>
size_t fused_smem_bytes(const ParamsT<T>& P)
{
    size_t b = 0;
    dispatch<T, Fused>(P, [&](auto f) { b = decltype(f)::L::bytes; return cudaSuccess; });
    return b;
}

template <typename T>
int fused_tiles(const ParamsT<T>& P)
{
    int n = 0;
    dispatch<T, Fused>(P, [&](auto f) { n = decltype(f)::tiles(P); return cudaSuccess; });
    return n;
}

template <typename T>
cudaError_t launch_courant_rates(const ParamsT<T>& P, unsigned char* rest, cudaStream_t s)
{
    return dispatch<T, Fused>(P, [&](auto f) { return decltype(f)::rates(P, rest, s); });
}

// One fused cycle: the Courant kernel (dt from the running maximum of the rates), the
// rest-tile kernel (copies the tiles at rest, queues the others), the persistent tile
// kernel.  With ev: an event before, one after the rest-tile kernel and one at the end.
template <typename T>
cudaError_t launch_step_fused(const ParamsT<T>& P, const OutPtrsT<T>& O, cudaStream_t s, cudaEvent_t* ev)
{
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_courant<T>(P, s);
    if (e == cudaSuccess) e = dispatch<T, Fused>(P, [&](auto f) { return decltype(f)::rest(P, O, s); });
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    e = dispatch<T, Fused>(P, [&](auto f) { return decltype(f)::launch(P, O, s); });
    if (ev) cudaEventRecord(ev[2], s);
    return e;
}

// ---- host side of the copy beside the tile kernel -----------------------------------------

TmaEncodeTiledFn tma_encode_tiled()
{
    static TmaEncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TmaEncodeTiledFn>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

namespace {

// the one instantiation whose tile-kernel CTA leaves room for a copy CTA on its SM (120
// registers a thread, 110 KB of shared memory): FP64, one hydrodynamic material, uniform grid
typedef Fused<double, 1, false, true> Beside;
constexpr int kBesideTW = Beside::S::TW, kBesideTH = Beside::S::TH, kBesideRegs = 120;
constexpr int kCopyStageBytes = 2 * kBesideTW * kBesideTH * 16 + kBesideTW * kBesideTH * 8;
constexpr int kCopySmemNeed = kCopyStages * kCopyStageBytes + kBesideTW * kBesideTH * 16 + 128;

// 2-D FP64 map: rows of `width` doubles `pitch` bytes apart, boxes of box_w x box_h
bool map_2d(CUtensorMap* map, const void* base, long width, long rows, long pitch, int box_w, int box_h)
{
    const TmaEncodeTiledFn fn = tma_encode_tiled();
    if (!fn || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 15) || width < 1 || rows < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool prepare_rest_copy(const ParamsT<double>& P, const OutPtrsT<double>& O, RestCopy* rc)
{
    if (!rc || P.nmat != 1 || P.any_strength || !P.uniform || (P.nr & 1)) return false;
    auto tile_k = k_step_fused<double, 1, false, true, kBesideTW, kBesideTH, Beside::S::NT, Beside::S::MINB, kBesideRegs>;
    auto copy_k = k_rest_copy<1, kBesideTW, kBesideTH>;
    auto scan_k = k_rest_scan<kBesideTW, kBesideTH>;
    cudaFuncAttributes ft, fc;
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0, optin = 0, reserved = 0;
    bool ok = cudaFuncGetAttributes(&ft, tile_k) == cudaSuccess && cudaFuncGetAttributes(&fc, copy_k) == cudaSuccess &&
              cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return false;
    }
    // registers are given out per warp in units of 256 (8 a thread), each warp's from the
    // quarter of the register file of its SM sub-partition (four a SM); the tile CTA's
    // warps spread evenly over the four, and the copy warp must fit beside them in one
    constexpr int kQuarters = 4;
    const int tile_warps = (Beside::S::NT / 32 + kQuarters - 1) / kQuarters;
    const int tile_regs = tile_warps * ((ft.numRegs + 7) / 8 * 8 * 32);
    const int copy_regs = (fc.numRegs + 7) / 8 * 8 * 32;
    if (tile_regs + copy_regs > regs_sm / kQuarters) return false;
    const int tile_smem = (int)Beside::L::bytes + (int)ft.sharedSizeBytes + reserved;
    // more than half of the SM: no SM takes two copy CTAs (which would leave no room there
    // for a tile CTA)
    int dyn = smem_sm / 2 - reserved - (int)fc.sharedSizeBytes + 128;
    dyn = ((dyn > kCopySmemNeed ? dyn : kCopySmemNeed) + 127) / 128 * 128;
    if (dyn > optin || tile_smem + dyn + (int)fc.sharedSizeBytes + reserved > smem_sm) return false;
    // the largest shared-memory share of the SM for all three kernels: an SM whose L1 /
    // shared split suits one of them alone would hold a second kernel's CTA back until it
    // drains
    int per_sm = 0, per_sm_tile = 0;
    const int maxshared = (int)cudaSharedmemCarveoutMaxShared;
    if (cudaFuncSetAttribute(copy_k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess ||
        cudaFuncSetAttribute(tile_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Beside::L::bytes) != cudaSuccess ||
        cudaFuncSetAttribute(copy_k, cudaFuncAttributePreferredSharedMemoryCarveout, maxshared) != cudaSuccess ||
        cudaFuncSetAttribute(tile_k, cudaFuncAttributePreferredSharedMemoryCarveout, maxshared) != cudaSuccess ||
        cudaFuncSetAttribute(scan_k, cudaFuncAttributePreferredSharedMemoryCarveout, maxshared) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, copy_k, 32, dyn) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tile, tile_k, Beside::S::NT, Beside::L::bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (per_sm != 1 || per_sm_tile != 1) return false;
    const long nr = P.nr, nz = P.nz;
    ok = map_2d(&rc->src[0], P.p.fr[0], 2 * nr, nz, 16 * nr, 2 * kBesideTW, kBesideTH) &&
         map_2d(&rc->src[1], P.p.I, nr, nz, 8 * nr, kBesideTW, kBesideTH) &&
         map_2d(&rc->src[2], P.p.eosc, 2 * nr, nz, 16 * nr, 2 * kBesideTW, kBesideTH) &&
         map_2d(&rc->dst[0], O.fr[0], 2 * nr, nz, 16 * nr, 2 * kBesideTW, kBesideTH) &&
         map_2d(&rc->dst[1], O.I, nr, nz, 8 * nr, kBesideTW, kBesideTH) &&
         map_2d(&rc->dst[2], O.eosc, 2 * nr, nz, 16 * nr, 2 * kBesideTW, kBesideTH) &&
         map_2d(&rc->v, O.v, 2 * (nr + 1), nz + 1, 16 * (nr + 1), 2 * kBesideTW, kBesideTH);
    if (!ok) return false;
    rc->ctas = sms;
    rc->smem = dyn;
    return true;
}

cudaError_t launch_step_fused_beside(const ParamsT<double>& P, const OutPtrsT<double>& O, const RestCopy& rc,
                                     cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join,
                                     cudaEvent_t* ev)
{
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_courant<double>(P, s);
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, fork, 0);
    if (e != cudaSuccess) return e;
    RestCopyArgs A;
    A.nr = P.nr; A.nz = P.nz; A.rest_in = O.rest_in; A.work = O.work; A.scal = P.p.scal; A.v = O.v;
    k_rest_copy<1, kBesideTW, kBesideTH><<<rc.ctas, 32, rc.smem, s2>>>(rc, A);
    e = cudaGetLastError();
    if (ev) cudaEventRecord(ev[1], s2);
    // the second stream joins back whatever happened, so that a capture stays well formed
    const cudaError_t ej = cudaEventRecord(join, s2);
    if (e == cudaSuccess) e = ej;
    if (e == cudaSuccess) {
        const int nt = Beside::tiles(P);
        k_rest_scan<kBesideTW, kBesideTH><<<(nt + kThreads - 1) / kThreads, kThreads, 0, s>>>(P.nr, P.nz, O);
        e = cudaGetLastError();
    }
    if (ev) cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) {
        k_step_fused<double, 1, false, true, kBesideTW, kBesideTH, Beside::S::NT, Beside::S::MINB, kBesideRegs>
            <<<O.ctas, Beside::S::NT, Beside::L::bytes, s>>>(P, O);
        e = cudaGetLastError();
    }
    if (ev) cudaEventRecord(ev[3], s);
    const cudaError_t ew = cudaStreamWaitEvent(s, join, 0);
    return e == cudaSuccess ? ew : e;
}

template cudaError_t prepare_fused<double>(const ParamsT<double>&, int*);
template cudaError_t prepare_fused<float>(const ParamsT<float>&, int*);
template int fused_tiles<double>(const ParamsT<double>&);
template int fused_tiles<float>(const ParamsT<float>&);
template size_t fused_smem_bytes<double>(const ParamsT<double>&);
template size_t fused_smem_bytes<float>(const ParamsT<float>&);
template cudaError_t launch_courant_rates<double>(const ParamsT<double>&, unsigned char*, cudaStream_t);
template cudaError_t launch_courant_rates<float>(const ParamsT<float>&, unsigned char*, cudaStream_t);
template cudaError_t launch_step_fused<double>(const ParamsT<double>&, const OutPtrsT<double>&, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_step_fused<float>(const ParamsT<float>&, const OutPtrsT<float>&, cudaStream_t, cudaEvent_t*);

}  // namespace salec
