// salec_api.cu -- host side of the C ABI in include/salec.h: state layout inside the
// caller's device buffer, initial conditions (layers, projectile, hydrostatic rows, PML
// profiles of Eq. 26, reference rows), stepping, field and scalar read-outs, checkpoint.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "salec_internal.cuh"
#include "salec_trace.h"

using namespace salec;

namespace {

constexpr size_t kAlign = 256;

// Block shapes the autotuner tries (threads in x are consecutive cells of a row, so x stays a
// multiple of the 32-thread warp); the smallest has 128 threads, which sizes the reduction
// partials.
const dim3 kShapes[] = {dim3(32, 4), dim3(32, 8), dim3(32, 16), dim3(64, 4), dim3(64, 8), dim3(128, 2), dim3(128, 4)};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
const dim3 kDefaultShape(32, 8);

// Offsets of every array inside the state buffer.  The persistent part (scalars, tables,
// fields, PML auxiliaries) comes first so a checkpoint is one contiguous range.
struct Layout {
    size_t es;   // bytes of one element of the form (8 FP64, 4 mixed); energies are always 8
    size_t scal, rR, rc, A_Z, invAZ, inv2rc, dr, idr, dz, idz, zc, A_R, V, invV, p0, rho_ref, I_ref, dB_c, dB_v, dR_c, dR_v;
    size_t pmax;
    // the fields a step rewrites, contiguous from pp_begin to persist_end (the fused form
    // reads one copy and writes the other: the second copy starts at pp_alt)
    size_t fr[kMaxMat], I, s01, s2d, v;
    size_t pb_c, pb_psi2, pb_v, pr_c, pr_psi2, pr_v;
    size_t pp_begin, persist_end;
    size_t pp_alt;
    size_t PM, pbphi, vL, mv, dK, kheat, frL[kMaxMat], VL, IL, sL01, sL2d, dMR, dMZ, partial, tmp;
    size_t eosc[2];   // the fused form's equation-of-state cache, one per copy of the fields
    size_t rest[2];   // the fused form's rest flags of the tiles, one per copy
    size_t work;      // two TileWork queues (one per copy the step reads)
    size_t list;      // the queued tiles
    size_t ntiles;    // bound on the fused form's tile count
    size_t total;
};

size_t take(size_t& cur, size_t bytes)
{
    const size_t off = cur;
    cur += (bytes + kAlign - 1) / kAlign * kAlign;
    return off;
}

Layout make_layout(const salec_grid& g, int precision)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    const size_t nr = g.nr, nz = g.nz, nc = nr * nz, nv = (nr + 1) * (nz + 1);
    const size_t pb = g.pml_bottom, pr = g.pml_right;
    L.es = precision == SALEC_FP32MIX ? sizeof(float) : sizeof(double);
    const size_t d = L.es, d2 = 2 * d, d4 = 4 * d, e8 = sizeof(double);
    size_t cur = 0;
    L.scal = take(cur, sizeof(DevScalars));
    L.rR = take(cur, (nr + 1) * d);
    L.rc = take(cur, nr * d);
    L.A_Z = take(cur, nr * d);
    L.invAZ = take(cur, nr * d);
    L.inv2rc = take(cur, nr * d);
    L.dr = take(cur, nr * d);
    L.idr = take(cur, nr * d);
    L.dz = take(cur, nz * d);
    L.idz = take(cur, nz * d);
    L.zc = take(cur, nz * e8);
    L.A_R = take(cur, (nr + 1) * d);
    L.V = take(cur, nr * d);
    L.invV = take(cur, nr * d);
    L.p0 = take(cur, nz * d);
    L.rho_ref = take(cur, nz * d);
    L.I_ref = take(cur, nz * e8);
    L.dB_c = take(cur, nz * d);
    L.dB_v = take(cur, (nz + 1) * d);
    L.dR_c = take(cur, nr * d);
    L.dR_v = take(cur, (nr + 1) * d);
    L.pmax = take(cur, nc * d);
    L.pp_begin = cur;
    for (int m = 0; m < g.nmat; ++m) L.fr[m] = take(cur, nc * d2);
    L.I = take(cur, nc * e8);
    L.s01 = take(cur, nc * d2);
    L.s2d = take(cur, nc * d2);
    L.v = take(cur, nv * d2);
    L.pb_c = take(cur, nr * pb * d2);
    L.pb_psi2 = take(cur, nr * pb * d);
    L.pb_v = take(cur, (nr + 1) * pb * d4);
    L.pr_c = take(cur, pr * nz * d2);
    L.pr_psi2 = take(cur, pr * nz * d);
    L.pr_v = take(cur, pr * (nz + 1) * d4);
    L.persist_end = cur;
    L.pp_alt = take(cur, L.persist_end - L.pp_begin);
    L.PM = take(cur, nc * d2);
    L.pbphi = take(cur, nc * d2);
    L.vL = take(cur, nv * d2);
    L.mv = take(cur, nv * d);
    L.dK = take(cur, nv * d);
    L.kheat = take(cur, nv * d);
    for (int m = 0; m < g.nmat; ++m) L.frL[m] = take(cur, nc * d2);
    L.VL = take(cur, nc * d);
    L.IL = take(cur, nc * e8);
    L.sL01 = take(cur, nc * d2);
    L.sL2d = take(cur, nc * d2);
    L.dMR = take(cur, (nr + 1) * nz * d);
    L.dMZ = take(cur, nr * (nz + 1) * d);
    L.eosc[0] = take(cur, nc * d2);
    L.eosc[1] = take(cur, nc * d2);
    L.ntiles = (size_t)((nr + kFusedTileW - 1) / kFusedTileW) * ((nz + kFusedTileMinH - 1) / kFusedTileMinH);
    L.rest[0] = take(cur, L.ntiles);
    L.rest[1] = take(cur, L.ntiles);
    L.work = take(cur, 2 * sizeof(TileWork));
    L.list = take(cur, L.ntiles * sizeof(int));
    size_t nb = 0;
    for (int k = 0; k < kNumShapes; ++k) {
        const size_t t = (size_t)tiles_of(g.nr, g.nz, 0, kShapes[k]);
        nb = t > nb ? t : nb;
    }
    const size_t nbv = (size_t)vertex_blocks(g.nr, g.nz);
    L.partial = take(cur, (nb > 4 * nbv ? nb : 4 * nbv) * e8);
    L.tmp = take(cur, nv * e8);
    L.total = cur;
    return L;
}

bool grid_ok(const salec_grid* g)
{
    if (!g) return false;
    if (g->nr < 1 || g->nz < 1 || g->nmat < 1 || g->nmat > kMaxMat) return false;
    if (!(g->dx > 0.0) || !(g->cfl > 0.0) || !(g->dt_growth > 0.0) || !(g->dt_max > 0.0)) return false;
    if (g->pml_right < 0 || g->pml_right >= g->nr || g->pml_bottom < 0 || g->pml_bottom >= g->nz) return false;
    if (g->f_min < 0.0 || g->gravity < 0.0) return false;
    if (g->bc_top != SALEC_TOP_OUTFLOW && g->bc_top != SALEC_TOP_WALL) return false;
    if (g->bc_bottom != SALEC_BOTTOM_NOSLIP && g->bc_bottom != SALEC_BOTTOM_FREESLIP) return false;
    if ((size_t)g->nr * (size_t)g->nz > (size_t)1 << 31) return false;
    return true;
}

}  // namespace

struct salec_ctx {
    salec_grid g;
    int precision;
    Layout L;
    char* base;
    size_t bytes;
    cudaStream_t stream;
    salec_material mats[kMaxMat];
    bool mat_set[kMaxMat];
    bool finalized;
    ParamsT<double> Pd;     // FP64 form
    ParamsT<float> Pf;      // mixed form
    dim3 shape[6];          // block shape of each kernel (salec_autotune picks them)
    // set-up accumulators (host, freed at finalize)
    std::vector<double> sV[kMaxMat], sM[kMaxMat], sE, sPz;
    std::vector<double> sR[kMaxMat];      // density shared by all contributions (exact)
    std::vector<char> sMix[kMaxMat];      // contributions of differing density
    std::vector<double> sI;               // specific energy shared by all contributions
    std::vector<char> sImix;
    std::vector<double> hydP, hydR;       // rows filled by a hydrostatic layer: pressure, density
    // geometry (per radian): column widths dr, vertex radii rR (nr+1), centre radii rc,
    // vertical face areas A_Z = rc dr; row heights dz, vertex heights zv (nz+1).  Cell
    // (i,j) has volume A_Z[i] dz[j]; the radial face at r_i of row j area rR[i] dz[j].
    std::vector<double> dr, rR, rc, A_Z, dz, zv;
    bool has_content = false;             // a layer or projectile is in: the spacing is fixed
    bool uniform = true;                  // every cell dx square
    double vol(int i, int j) const { return A_Z[i] * dz[j]; }
    std::string err;
    // stepping in CUDA-graph replays of kGraphChunk steps (captured once per block-shape
    // set; false after a capture failed, then plain launches)
    cudaGraphExec_t graph = nullptr;
    dim3 graph_shape[6];
    bool graph_ok = true;
    // step form: SALEC_STEP_FUSED (Courant kernel + one tile kernel, ping-pong copies of the
    // rewritten fields) or SALEC_STEP_PHASES (seven launches, in place)
    int form = SALEC_STEP_PHASES;
    int parity = 0;                       // 1: the current fields are in the second copy
    bool rates_valid = false;             // the running Courant maximum holds the current state's rates
    ParamsT<double> Pd_alt;               // the FP64 / mixed parameters reading the second copy
    ParamsT<float> Pf_alt;
    OutPtrsT<double> Od[2];               // where a fused step from copy k writes (the other copy)
    OutPtrsT<float> Of[2];
    cudaGraphExec_t fgraph[2] = {nullptr, nullptr};   // fused chunks starting from copy 0 / 1
    bool fgraph_ok = true;
    bool rest_copy = true;                // tiles at rest copied (salec_set_rest_copy)
    bool copy_beside = false;             // ... by the copy kernel beside the tile kernel, where available
    RestCopy* rcopy = nullptr;            // its maps and launch shape for steps from copy 0 / 1 (FP64 form)
    cudaStream_t s2 = nullptr;            // its stream, and the events that fork it off and join it back
    cudaEvent_t fork = nullptr, join = nullptr;
    // optional per-kernel timing: 7 events per recorded step
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
};

static salec_status fail(salec_ctx* ctx, salec_status st, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

static salec_status cuda_check(salec_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return SALEC_OK;
    return fail(ctx, SALEC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <typename T>
static T* at(salec_ctx* ctx, size_t off) { return reinterpret_cast<T*>(ctx->base + off); }

template <typename T>
static void fill_params(salec_ctx* ctx, ParamsT<T>& P)
{
    typedef typename VT<T>::T2 T2;
    typedef typename VT<T>::T4 T4;
    const salec_grid& g = ctx->g;
    const Layout& L = ctx->L;
    P.nr = g.nr; P.nz = g.nz; P.nmat = g.nmat; P.pr = g.pml_right; P.pb = g.pml_bottom;
    P.bc_top = g.bc_top; P.bc_bottom = g.bc_bottom;
    P.any_strength = 0;
    for (int m = 0; m < g.nmat; ++m) {
        P.mat[m] = to_mat<T>(ctx->mats[m]);
        if (ctx->mats[m].strength == SALEC_STRENGTH_COLLINS) P.any_strength = 1;
    }
    P.nblk_cells = cell_blocks(g.nr, g.nz);
    P.cfl = T(g.cfl); P.g = T(g.gravity); P.cq = T(g.av_cq);
    P.cl = T(g.av_cl); P.f_min = T(g.f_min);
    P.uniform = ctx->uniform ? 1 : 0;
    P.dx = T(g.dx); P.dx2 = T(g.dx * g.dx); P.idx = T(1.0 / g.dx); P.dxd = g.dx;
    P.cfld = g.cfl; P.growth = g.dt_growth; P.dt_max = g.dt_max; P.dt_min = g.dt_min;
    PtrsT<T>& p = P.p;
    for (int m = 0; m < kMaxMat; ++m) {
        p.fr[m] = m < g.nmat ? at<T2>(ctx, L.fr[m]) : nullptr;
        p.frL[m] = m < g.nmat ? at<T2>(ctx, L.frL[m]) : nullptr;
    }
    p.I = at<double>(ctx, L.I); p.s01 = at<T2>(ctx, L.s01); p.s2d = at<T2>(ctx, L.s2d);
    p.pmax = at<T>(ctx, L.pmax); p.v = at<T2>(ctx, L.v);
    p.pb_c = at<T2>(ctx, L.pb_c); p.pb_psi2 = at<T>(ctx, L.pb_psi2); p.pb_v = at<T4>(ctx, L.pb_v);
    p.pr_c = at<T2>(ctx, L.pr_c); p.pr_psi2 = at<T>(ctx, L.pr_psi2); p.pr_v = at<T4>(ctx, L.pr_v);
    p.rR = at<T>(ctx, L.rR); p.rc = at<T>(ctx, L.rc); p.A_Z = at<T>(ctx, L.A_Z); p.invAZ = at<T>(ctx, L.invAZ);
    p.inv2rc = at<T>(ctx, L.inv2rc); p.dr = at<T>(ctx, L.dr); p.idr = at<T>(ctx, L.idr);
    p.dz = at<T>(ctx, L.dz); p.idz = at<T>(ctx, L.idz); p.zc = at<double>(ctx, L.zc); p.p0 = at<T>(ctx, L.p0);
    p.A_R = at<T>(ctx, L.A_R); p.V = at<T>(ctx, L.V); p.invV = at<T>(ctx, L.invV);
    p.rho_ref = at<T>(ctx, L.rho_ref); p.I_ref = at<double>(ctx, L.I_ref); p.dB_c = at<T>(ctx, L.dB_c);
    p.dB_v = at<T>(ctx, L.dB_v); p.dR_c = at<T>(ctx, L.dR_c); p.dR_v = at<T>(ctx, L.dR_v);
    p.PM = at<T2>(ctx, L.PM); p.pbphi = at<T2>(ctx, L.pbphi); p.vL = at<T2>(ctx, L.vL);
    p.mv = at<T>(ctx, L.mv); p.dK = at<T>(ctx, L.dK); p.kheat = at<T>(ctx, L.kheat);
    p.VL = at<T>(ctx, L.VL); p.IL = at<double>(ctx, L.IL); p.sL01 = at<T2>(ctx, L.sL01);
    p.sL2d = at<T2>(ctx, L.sL2d); p.dMR = at<T>(ctx, L.dMR); p.dMZ = at<T>(ctx, L.dMZ);
    p.eosc = at<T2>(ctx, L.eosc[0]);
    p.partial = at<double>(ctx, L.partial);
    p.scal = at<DevScalars>(ctx, L.scal);
}

static bool mixed(const salec_ctx* ctx) { return ctx->precision == SALEC_FP32MIX; }

// The same parameters with the rewritten fields read from the second copy, and the output
// pointers of a fused step from copy 0 (writes copy 1) and from copy 1 (writes copy 0).
template <typename T>
static void fill_pingpong(salec_ctx* ctx, const ParamsT<T>& P0, ParamsT<T>& P1, OutPtrsT<T>* O)
{
    typedef typename VT<T>::T2 T2;
    typedef typename VT<T>::T4 T4;
    const Layout& L = ctx->L;
    const size_t shift = L.pp_alt - L.pp_begin;
    auto copy_at = [&](int k, size_t off) { return k == 0 ? off : off + shift; };
    P1 = P0;
    for (int m = 0; m < kMaxMat; ++m) P1.p.fr[m] = m < ctx->g.nmat ? at<T2>(ctx, copy_at(1, L.fr[m])) : nullptr;
    P1.p.I = at<double>(ctx, copy_at(1, L.I));
    P1.p.s01 = at<T2>(ctx, copy_at(1, L.s01)); P1.p.s2d = at<T2>(ctx, copy_at(1, L.s2d));
    P1.p.v = at<T2>(ctx, copy_at(1, L.v));
    P1.p.pb_c = at<T2>(ctx, copy_at(1, L.pb_c)); P1.p.pb_psi2 = at<T>(ctx, copy_at(1, L.pb_psi2));
    P1.p.pb_v = at<T4>(ctx, copy_at(1, L.pb_v));
    P1.p.pr_c = at<T2>(ctx, copy_at(1, L.pr_c)); P1.p.pr_psi2 = at<T>(ctx, copy_at(1, L.pr_psi2));
    P1.p.pr_v = at<T4>(ctx, copy_at(1, L.pr_v));
    P1.p.eosc = at<T2>(ctx, L.eosc[1]);
    for (int k = 0; k < 2; ++k) {
        const int w = 1 - k;      // a step from copy k writes copy 1 - k
        OutPtrsT<T>& o = O[k];
        memset(&o, 0, sizeof(o));
        for (int m = 0; m < ctx->g.nmat; ++m) o.fr[m] = at<T2>(ctx, copy_at(w, L.fr[m]));
        o.I = at<double>(ctx, copy_at(w, L.I));
        o.s01 = at<T2>(ctx, copy_at(w, L.s01)); o.s2d = at<T2>(ctx, copy_at(w, L.s2d));
        o.v = at<T2>(ctx, copy_at(w, L.v));
        o.pb_c = at<T2>(ctx, copy_at(w, L.pb_c)); o.pb_psi2 = at<T>(ctx, copy_at(w, L.pb_psi2));
        o.pb_v = at<T4>(ctx, copy_at(w, L.pb_v));
        o.pr_c = at<T2>(ctx, copy_at(w, L.pr_c)); o.pr_psi2 = at<T>(ctx, copy_at(w, L.pr_psi2));
        o.pr_v = at<T4>(ctx, copy_at(w, L.pr_v));
        o.eosc = at<T2>(ctx, L.eosc[w]);
        o.rest_in = at<unsigned char>(ctx, L.rest[k]);
        o.rest_out = at<unsigned char>(ctx, L.rest[w]);
        o.work = at<TileWork>(ctx, L.work) + k;
        o.work_next = at<TileWork>(ctx, L.work) + w;
        o.list = at<int>(ctx, L.list);
    }
}

// Bring the current fields (and the equation-of-state cache and the rest flags that go with
// them) into the first copy, where every read-out, checkpoint, batch and the phase kernels
// find them, after an odd number of fused steps: three device copies; the queue the step
// that wrote the second copy used moves to the second copy's place (salec_fused_queue reads
// it there) and the first copy's is emptied for the next step.
static cudaError_t canonical(salec_ctx* ctx)
{
    if (ctx->parity == 0) return cudaSuccess;
    const Layout& L = ctx->L;
    cudaError_t e = cudaMemcpyAsync(ctx->base + L.pp_begin, ctx->base + L.pp_alt, L.persist_end - L.pp_begin,
                                    cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->base + L.eosc[0], ctx->base + L.eosc[1], L.eosc[1] - L.eosc[0], cudaMemcpyDeviceToDevice,
                            ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->base + L.rest[0], ctx->base + L.rest[1], L.ntiles, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->base + L.work + sizeof(TileWork), ctx->base + L.work, sizeof(TileWork),
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->base + L.work, 0, sizeof(TileWork), ctx->stream);
    if (e == cudaSuccess) ctx->parity = 0;
    return e;
}

// vertex positions, centre radii and vertical face areas from the cell sizes, summed
// outward from the axis and up from the bottom
static void set_geometry(salec_ctx* ctx)
{
    const int nr = ctx->g.nr, nz = ctx->g.nz;
    ctx->rR.assign(nr + 1, 0.0);
    ctx->rc.assign(nr, 0.0);
    ctx->A_Z.assign(nr, 0.0);
    ctx->zv.assign(nz + 1, 0.0);
    for (int i = 0; i < nr; ++i) ctx->rR[i + 1] = ctx->rR[i] + ctx->dr[i];
    for (int i = 0; i < nr; ++i) {
        ctx->rc[i] = 0.5 * (ctx->rR[i] + ctx->rR[i + 1]);
        ctx->A_Z[i] = ctx->rc[i] * ctx->dr[i];
    }
    for (int j = 0; j < nz; ++j) ctx->zv[j + 1] = ctx->zv[j] + ctx->dz[j];
    bool uni = true;
    for (int i = 0; i < nr; ++i) uni = uni && ctx->dr[i] == ctx->g.dx;
    for (int j = 0; j < nz; ++j) uni = uni && ctx->dz[j] == ctx->g.dx;
    ctx->uniform = uni;
}

extern "C" {

salec_status salec_state_bytes(const salec_grid* grid, int precision, size_t* bytes)
{
    if (!grid_ok(grid) || (precision != SALEC_FP64 && precision != SALEC_FP32MIX) || !bytes) return SALEC_EINVAL;
    *bytes = make_layout(*grid, precision).total;
    return SALEC_OK;
}

salec_status salec_create(const salec_grid* grid, int precision, void* dev_state, size_t bytes, void* stream,
                          salec_ctx** out)
{
    if (!out || !grid_ok(grid) || (precision != SALEC_FP64 && precision != SALEC_FP32MIX)) return SALEC_EINVAL;
    if (precision == SALEC_FP32MIX && !(grid->f_min >= 1e-7)) return SALEC_EINVAL;   // FP32 fractions need a floor
    Layout L = make_layout(*grid, precision);
    if (!dev_state || bytes < L.total || ((uintptr_t)dev_state % kAlign) != 0) return SALEC_ENOMEM;
    salec_ctx* ctx = new salec_ctx();
    ctx->g = *grid;
    ctx->precision = precision;
    ctx->L = L;
    ctx->base = (char*)dev_state;
    ctx->bytes = bytes;
    ctx->stream = (cudaStream_t)stream;
    memset(ctx->mats, 0, sizeof(ctx->mats));
    for (int m = 0; m < kMaxMat; ++m) ctx->mat_set[m] = false;
    ctx->finalized = false;
    for (int k = 0; k < 6; ++k) ctx->shape[k] = kDefaultShape;
    const size_t nc = (size_t)grid->nr * grid->nz;
    for (int m = 0; m < grid->nmat; ++m) {
        ctx->sV[m].assign(nc, 0.0); ctx->sM[m].assign(nc, 0.0);
        ctx->sR[m].assign(nc, 0.0); ctx->sMix[m].assign(nc, 0);
    }
    ctx->sE.assign(nc, 0.0);
    ctx->sI.assign(nc, 0.0);
    ctx->sImix.assign(nc, 0);
    ctx->sPz.assign(nc, 0.0);
    ctx->hydP.assign(grid->nz, 0.0);
    ctx->hydR.assign(grid->nz, 0.0);
    // uniform cells of dx until salec_set_spacing
    ctx->dr.assign(grid->nr, grid->dx);
    ctx->dz.assign(grid->nz, grid->dx);
    set_geometry(ctx);
    *out = ctx;
    return SALEC_OK;
}

salec_status salec_set_spacing(salec_ctx* ctx, const double* dr, const double* dz)
{
    if (!ctx || !dr || !dz) return SALEC_EINVAL;
    if (ctx->finalized || ctx->has_content)
        return fail(ctx, SALEC_EORDER, "set_spacing after a layer, projectile or finalize");
    for (int i = 0; i < ctx->g.nr; ++i)
        if (!(dr[i] > 0.0) || !std::isfinite(dr[i])) return fail(ctx, SALEC_EINVAL, "dr[%d] must be positive", i);
    for (int j = 0; j < ctx->g.nz; ++j)
        if (!(dz[j] > 0.0) || !std::isfinite(dz[j])) return fail(ctx, SALEC_EINVAL, "dz[%d] must be positive", j);
    ctx->dr.assign(dr, dr + ctx->g.nr);
    ctx->dz.assign(dz, dz + ctx->g.nz);
    set_geometry(ctx);
    return SALEC_OK;
}

salec_status salec_set_material(salec_ctx* ctx, int id, const salec_material* mat)
{
    if (!ctx || !mat) return SALEC_EINVAL;
    if (ctx->finalized) return fail(ctx, SALEC_EORDER, "set_material after finalize");
    if (id < 0 || id >= ctx->g.nmat) return fail(ctx, SALEC_EINVAL, "material id %d out of range", id);
    if (mat->eos != SALEC_EOS_TILLOTSON && mat->eos != SALEC_EOS_IDEAL_GAS)
        return fail(ctx, SALEC_EINVAL, "unknown eos %d", mat->eos);
    if (!(mat->rho0 > 0.0)) return fail(ctx, SALEC_EINVAL, "rho0 must be positive");
    if (mat->eos == SALEC_EOS_TILLOTSON && !(mat->E0 > 0.0 && mat->A > 0.0 && mat->Ecv > mat->Eiv))
        return fail(ctx, SALEC_EINVAL, "Tillotson constants out of range");
    if (mat->strength != SALEC_STRENGTH_NONE && mat->strength != SALEC_STRENGTH_COLLINS)
        return fail(ctx, SALEC_EINVAL, "unknown strength model %d", mat->strength);
    if (mat->strength == SALEC_STRENGTH_COLLINS && !(mat->G > 0.0 && mat->Yim > mat->Yi0 && mat->eps_fb > 0.0))
        return fail(ctx, SALEC_EINVAL, "strength constants out of range");
    ctx->mats[id] = *mat;
    ctx->mat_set[id] = true;
    return SALEC_OK;
}

// Add volume `vol` of material `mat` at density rho to cell c.  Cells whose contributions
// share one density keep it exactly; otherwise the density is mass / volume.
static void add_content(salec_ctx* ctx, int mat, size_t c, double vol, double rho, double I0, double vz)
{
    const double mass = rho * vol;
    bool empty = true;
    for (int m = 0; m < ctx->g.nmat; ++m) empty = empty && ctx->sV[m][c] == 0.0;
    if (empty) ctx->sI[c] = I0;
    else if (ctx->sI[c] != I0) ctx->sImix[c] = 1;
    if (ctx->sV[mat][c] == 0.0) ctx->sR[mat][c] = rho;
    else if (ctx->sR[mat][c] != rho) ctx->sMix[mat][c] = 1;
    ctx->sV[mat][c] += vol;
    ctx->sM[mat][c] += mass;
    ctx->sE[c] += mass * I0;
    ctx->sPz[c] += mass * vz;
}

salec_status salec_add_layer(salec_ctx* ctx, int mat, double zlo, double zhi, double rho, double I0, double vz)
{
    if (!ctx) return SALEC_EINVAL;
    if (ctx->finalized) return fail(ctx, SALEC_EORDER, "add_layer after finalize");
    if (mat < 0 || mat >= ctx->g.nmat || !ctx->mat_set[mat]) return fail(ctx, SALEC_EORDER, "material %d not set", mat);
    if (!(zhi > zlo)) return fail(ctx, SALEC_EINVAL, "layer needs zlo < zhi");
    const salec_material& M = ctx->mats[mat];
    const int nr = ctx->g.nr, nz = ctx->g.nz;
    const double g = ctx->g.gravity;
    const bool hydro = rho <= 0.0 && g > 0.0 && M.eos == SALEC_EOS_TILLOTSON;
    if (hydro && I0 != 0.0) return fail(ctx, SALEC_EINVAL, "hydrostatic layer must be cold (I0 = 0)");
    ctx->has_content = true;
    std::vector<double> w(nz), rrow(nz, rho > 0.0 ? rho : M.rho0);
    for (int j = 0; j < nz; ++j) {
        const double z0 = ctx->zv[j], z1 = ctx->zv[j + 1];
        const double lo = zlo > z0 ? zlo : z0, hi = zhi < z1 ? zhi : z1;
        // a row inside the layer is full (z1 - z0 need not round to dz exactly)
        w[j] = (zlo <= z0 && zhi >= z1) ? 1.0 : (hi > lo ? (hi - lo) / ctx->dz[j] : 0.0);
    }
    if (hydro) {
        // discrete hydrostatic balance at the vertex between rows j (below) and j+1:
        // P_j - P_{j+1} = g (rho_j dz_j + rho_{j+1} dz_{j+1}) / 2 with the cold curve
        // P = A mu + B mu^2; per row a quadratic in mu, solved in the cancellation-free form
        // of its root.  Wup is the upper half cell's weight g rho_{j+1} dz_{j+1} / 2.
        // A layer right below the rows of an earlier hydrostatic layer carries their
        // weight: it starts from the pressure and density of the row above it.
        for (int j = 0; j < nz; ++j)
            if (w[j] > 0.0 && w[j] < 1.0) return fail(ctx, SALEC_EINVAL, "hydrostatic layer must fill whole rows");
        double Pup = 0.0, Wup = 0.0;
        int j = nz - 1;
        while (j >= 0 && !(w[j] > 0.0)) --j;
        if (j >= 0 && j + 1 < nz && ctx->hydR[j + 1] > 0.0) {
            Pup = ctx->hydP[j + 1];
            Wup = (0.5 * ctx->dz[j + 1] * g) * ctx->hydR[j + 1];
        }
        for (; j >= 0 && w[j] > 0.0; --j) {
            const double k = 0.5 * ctx->dz[j] * g;
            const double rhs = Pup + Wup;
            const double lin = M.A - k * M.rho0, cst = k * M.rho0 + rhs;
            double mu;
            if (M.B != 0.0) mu = 2.0 * cst / (lin + sqrt(lin * lin + 4.0 * M.B * cst));
            else mu = cst / lin;
            rrow[j] = M.rho0 * (1.0 + mu);
            Pup = M.A * mu + M.B * mu * mu;
            Wup = k * rrow[j];
            ctx->hydP[j] = Pup;
            ctx->hydR[j] = rrow[j];
        }
    }
    for (int j = 0; j < nz; ++j) {
        if (!(w[j] > 0.0)) continue;
        for (int i = 0; i < nr; ++i) {
            add_content(ctx, mat, (size_t)j * nr + i, w[j] * ctx->vol(i, j), rrow[j], I0, vz);
        }
    }
    return SALEC_OK;
}

salec_status salec_place_projectile(salec_ctx* ctx, int mat, double radius, double zc, double vz, double rho, double I0)
{
    if (!ctx) return SALEC_EINVAL;
    if (ctx->finalized) return fail(ctx, SALEC_EORDER, "place_projectile after finalize");
    if (mat < 0 || mat >= ctx->g.nmat || !ctx->mat_set[mat]) return fail(ctx, SALEC_EORDER, "material %d not set", mat);
    if (!(radius > 0.0)) return fail(ctx, SALEC_EINVAL, "radius must be positive");
    const double r0 = rho > 0.0 ? rho : ctx->mats[mat].rho0;
    const int nr = ctx->g.nr, nz = ctx->g.nz;
    const double R2 = radius * radius;
    ctx->has_content = true;
    // only rows and columns that can touch the sphere
    for (int j = 0; j < nz; ++j) {
        if (ctx->zv[j + 1] < zc - radius || ctx->zv[j] > zc + radius) continue;
        for (int i = 0; i < nr && ctx->rR[i] <= radius; ++i) {
            double wi = 0.0, wt = 0.0;
            for (int b = 0; b < 16; ++b) {
                const double zs = ctx->zv[j] + ctx->dz[j] * (((double)b + 0.5) / 16.0);
                const double dz = zs - zc;
                for (int a = 0; a < 16; ++a) {
                    const double rs = ctx->rR[i] + ctx->dr[i] * (((double)a + 0.5) / 16.0);
                    wt += rs;
                    if (rs * rs + dz * dz < R2) wi += rs;
                }
            }
            const double frac = wi / wt;
            if (!(frac > 0.0)) continue;
            const size_t c = (size_t)j * nr + i;
            const double keep = 1.0 - frac;
            for (int k = 0; k < ctx->g.nmat; ++k) { ctx->sV[k][c] *= keep; ctx->sM[k][c] *= keep; }
            ctx->sE[c] *= keep;
            ctx->sPz[c] *= keep;
            add_content(ctx, mat, c, frac * ctx->vol(i, j), r0, I0, vz);
        }
    }
    return SALEC_OK;
}

// Eq. 26: d(y) = 3 c / (2 delta) (y / delta)^2 log(1 / R), strip thickness delta and the
// distance y from its inner edge in metres
static double profile(double c, double delta, double y, double R)
{
    if (!(delta > 0.0) || y <= 0.0) return 0.0;
    const double s = y / delta;
    return 1.5 * c / delta * s * s * log(1.0 / R);
}

// The FP64 form's copy of the tiles at rest beside the tile kernel: maps, stream and events,
// where the grid and the device allow it (otherwise the rest-tile kernel copies them).
static void release_beside(salec_ctx* ctx)
{
    delete[] ctx->rcopy;
    ctx->rcopy = nullptr;
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->s2) cudaStreamDestroy(ctx->s2);
    ctx->fork = ctx->join = nullptr;
    ctx->s2 = nullptr;
}

static void prepare_beside(salec_ctx* ctx)
{
    release_beside(ctx);
    RestCopy* rc = new (std::nothrow) RestCopy[2];
    if (!rc) return;
    if (!prepare_rest_copy(ctx->Pd, ctx->Od[0], &rc[0]) || !prepare_rest_copy(ctx->Pd_alt, ctx->Od[1], &rc[1])) {
        delete[] rc;
        return;
    }
    if (cudaStreamCreateWithFlags(&ctx->s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        delete[] rc;
        release_beside(ctx);
        return;
    }
    ctx->rcopy = rc;
}

// a fused step copies its tiles at rest beside the tile kernel
static bool beside(const salec_ctx* ctx) { return ctx->rest_copy && ctx->copy_beside && ctx->rcopy && !mixed(ctx); }

// events one recorded step takes, and the pair that brackets timed kernel k
static int events_per_step(const salec_ctx* ctx)
{
    if (ctx->form != SALEC_STEP_FUSED) return launches_per_step() + 1;
    return beside(ctx) ? 4 : 3;
}

static void kernel_events(const salec_ctx* ctx, int k, int* a, int* b)
{
    const bool two = ctx->form == SALEC_STEP_FUSED && beside(ctx);
    *a = two ? 2 * k : k;
    *b = *a + 1;
}

salec_status salec_finalize(salec_ctx* ctx)
{
    if (!ctx) return SALEC_EINVAL;
    if (ctx->finalized) return fail(ctx, SALEC_EORDER, "finalize called twice");
    const salec_grid& g = ctx->g;
    for (int m = 0; m < g.nmat; ++m)
        if (!ctx->mat_set[m]) return fail(ctx, SALEC_EORDER, "material %d not set", m);
    const int nr = g.nr, nz = g.nz, pr = g.pml_right, pb = g.pml_bottom;
    const size_t nc = (size_t)nr * nz, nv = (size_t)(nr + 1) * (nz + 1);
    fill_params<double>(ctx, ctx->Pd);
    fill_params<float>(ctx, ctx->Pf);
    const ParamsT<double>& P = ctx->Pd;
    // PML wave speed
    double c = g.pml_c;
    if (!(c > 0.0)) {
        c = 0.0;
        for (int m = 0; m < g.nmat; ++m)
            if (ctx->mats[m].eos == SALEC_EOS_TILLOTSON) {
                const double cm = sqrt(ctx->mats[m].A / ctx->mats[m].rho0);
                c = cm > c ? cm : c;
            }
    }
    if ((pr > 0 || pb > 0) && !(c > 0.0 && g.pml_R > 0.0 && g.pml_R < 1.0))
        return fail(ctx, SALEC_EINVAL, "PML needs a wave speed and 0 < R < 1");
    if (!(g.pml_alpha >= 0.0)) return fail(ctx, SALEC_EINVAL, "pml_alpha must be >= 0");
    // auxiliaries relax at alpha = pml_alpha c / delta of their strip (complex-frequency-
    // shifted stretch 1 + d / (alpha + i omega)), so a static tangential term cannot grow them
    // without bound
    const double delta_b = ctx->zv[pb], r_in = ctx->rR[nr - pr], delta_r = ctx->rR[nr] - r_in;
    const double ab = pb > 0 ? g.pml_alpha * c / delta_b : 0.0, ar = pr > 0 ? g.pml_alpha * c / delta_r : 0.0;
    ctx->Pd.alpha_b = ab; ctx->Pd.alpha_r = ar;
    ctx->Pf.alpha_b = (float)ab; ctx->Pf.alpha_r = (float)ar;
    // cells
    std::vector<double2> fr[kMaxMat];
    for (int m = 0; m < g.nmat; ++m) fr[m].assign(nc, make_double2(0.0, 0.0));
    std::vector<double> I(nc, 0.0), Mkept(nc, 0.0), Mall(nc, 0.0);
    for (size_t cc = 0; cc < nc; ++cc) {
        const int i = (int)(cc % nr), jj = (int)(cc / nr);
        double mk = 0.0, ma = 0.0;
        for (int m = 0; m < g.nmat; ++m) {
            double f = ctx->sV[m][cc] / ctx->vol(i, jj);
            if (f < g.f_min) f = 0.0;
            ma += ctx->sM[m][cc];
            if (f > 0.0) {
                fr[m][cc] = make_double2(f, ctx->sMix[m][cc] ? ctx->sM[m][cc] / ctx->sV[m][cc] : ctx->sR[m][cc]);
                mk += ctx->sM[m][cc];
            }
        }
        Mkept[cc] = mk;
        Mall[cc] = ma;
        I[cc] = mk > 0.0 ? (ctx->sImix[cc] ? ctx->sE[cc] / mk : ctx->sI[cc]) : 0.0;
    }
    // vertices: quarter-cell momentum / quarter-cell mass
    std::vector<double2> v(nv, make_double2(0.0, 0.0));
    for (int j = 0; j <= nz; ++j)
        for (int i = 0; i <= nr; ++i) {
            double mom = 0.0, mass = 0.0;
            for (int dj = -1; dj <= 0; ++dj)
                for (int di = -1; di <= 0; ++di) {
                    const int ci = i + di, cj = j + dj;
                    if (ci < 0 || ci >= nr || cj < 0 || cj >= nz) continue;
                    const size_t cc = (size_t)cj * nr + ci;
                    if (Mall[cc] > 0.0) mom += 0.25 * ctx->sPz[cc] * (Mkept[cc] / Mall[cc]);
                    mass += 0.25 * Mkept[cc];
                }
            double vz = mass > 0.0 ? mom / mass : 0.0;
            if (j == 0 || (j == nz && g.bc_top == SALEC_TOP_WALL)) vz = 0.0;
            v[(size_t)j * (nr + 1) + i] = make_double2(0.0, vz);
        }
    // reference rows from the outermost column
    std::vector<double> p0(nz, 0.0), rref(nz, 0.0), Iref(nz, 0.0);
    for (int j = 0; j < nz; ++j) {
        const size_t cc = (size_t)j * nr + (nr - 1);
        double phat = 0.0, phi = 0.0, mass = 0.0;
        for (int m = 0; m < g.nmat; ++m) {
            const double2 f = fr[m][cc];
            if (!(f.x > 0.0)) continue;
            double pm, c2;
            eos_eval<double>(P.mat[m], f.y, I[cc], pm, c2);
            const double pmin = P.mat[m].p_t * expansion_weight(P.mat[m], f.y);
            pm = pm < pmin ? pmin : pm;
            phat += f.x * pm; phi += f.x; mass += f.x * f.y;
        }
        if (phi > 0.0) { p0[j] = phat / phi; rref[j] = mass / phi; Iref[j] = I[cc]; }
    }
    // PML profiles (Eq. 26)
    std::vector<double> dBc(nz, 0.0), dBv(nz + 1, 0.0), dRc(nr, 0.0), dRv(nr + 1, 0.0);
    for (int j = 0; j < pb; ++j) {
        dBc[j] = profile(c, delta_b, delta_b - (ctx->zv[j] + 0.5 * ctx->dz[j]), g.pml_R);
        dBv[j] = profile(c, delta_b, delta_b - ctx->zv[j], g.pml_R);
    }
    for (int i = nr - pr; i < nr; ++i) dRc[i] = profile(c, delta_r, ctx->rc[i] - r_in, g.pml_R);
    for (int i = nr - pr + 1; i <= nr; ++i) dRv[i] = profile(c, delta_r, ctx->rR[i] - r_in, g.pml_R);
    std::vector<double> invAZ(nr), inv2rc(nr), idr(nr), idz(nz), zcen(nz);
    // the uniform-grid tables (used when every cell is dx square): A_R = r_i dx,
    // V = r_c dx^2 with r_i = i dx and r_c = (i + 1/2) dx
    std::vector<double> uAR(nr + 1), uV(nr), uinvV(nr);
    for (int i = 0; i <= nr; ++i) uAR[i] = ((double)i * g.dx) * g.dx;
    for (int i = 0; i < nr; ++i) {
        uV[i] = (((double)i + 0.5) * g.dx) * g.dx * g.dx;
        uinvV[i] = 1.0 / uV[i];
    }
    for (int i = 0; i < nr; ++i) {
        invAZ[i] = 1.0 / ctx->A_Z[i];
        inv2rc[i] = 1.0 / (2.0 * ctx->rc[i]);
        idr[i] = 1.0 / ctx->dr[i];
    }
    for (int j = 0; j < nz; ++j) {
        idz[j] = 1.0 / ctx->dz[j];
        zcen[j] = ctx->zv[j] + 0.5 * ctx->dz[j];
    }
    // scalars
    DevScalars s;
    memset(&s, 0, sizeof(s));
    s.dt_prev = g.dt_init;
    s.t_end = 1e300;
    s.active = 1;
    const Layout& L = ctx->L;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(ctx->base, 0, L.persist_end, st);
    auto up = [&](size_t off, const void* src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(ctx->base + off, src, n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // src may be a temporary
    };
    // arrays of the form's element type: converted from FP64 on the host when mixed
    const bool mx = mixed(ctx);
    auto upT = [&](size_t off, const double* src, size_t n) {
        if (!mx) { up(off, src, n * sizeof(double)); return; }
        std::vector<float> f(n);
        for (size_t k = 0; k < n; ++k) f[k] = (float)src[k];
        up(off, f.data(), n * sizeof(float));
    };
    up(L.scal, &s, sizeof(s));
    upT(L.rR, ctx->rR.data(), nr + 1);
    upT(L.rc, ctx->rc.data(), nr);
    upT(L.A_Z, ctx->A_Z.data(), nr);
    upT(L.invAZ, invAZ.data(), nr);
    upT(L.inv2rc, inv2rc.data(), nr);
    upT(L.dr, ctx->dr.data(), nr);
    upT(L.idr, idr.data(), nr);
    upT(L.dz, ctx->dz.data(), nz);
    upT(L.idz, idz.data(), nz);
    up(L.zc, zcen.data(), nz * sizeof(double));
    upT(L.A_R, uAR.data(), nr + 1);
    upT(L.V, uV.data(), nr);
    upT(L.invV, uinvV.data(), nr);
    upT(L.p0, p0.data(), nz);
    upT(L.rho_ref, rref.data(), nz);
    up(L.I_ref, Iref.data(), nz * sizeof(double));
    upT(L.dB_c, dBc.data(), nz);
    upT(L.dB_v, dBv.data(), nz + 1);
    upT(L.dR_c, dRc.data(), nr);
    upT(L.dR_v, dRv.data(), nr + 1);
    for (int m = 0; m < g.nmat; ++m) upT(L.fr[m], reinterpret_cast<const double*>(fr[m].data()), 2 * nc);
    up(L.I, I.data(), nc * sizeof(double));
    upT(L.v, reinterpret_cast<const double*>(v.data()), 2 * nv);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "finalize upload");
    for (int m = 0; m < kMaxMat; ++m) {
        ctx->sV[m].clear(); ctx->sV[m].shrink_to_fit(); ctx->sM[m].clear(); ctx->sM[m].shrink_to_fit();
        ctx->sR[m].clear(); ctx->sR[m].shrink_to_fit(); ctx->sMix[m].clear(); ctx->sMix[m].shrink_to_fit();
    }
    ctx->sE.clear(); ctx->sE.shrink_to_fit(); ctx->sPz.clear(); ctx->sPz.shrink_to_fit();
    ctx->sI.clear(); ctx->sI.shrink_to_fit(); ctx->sImix.clear(); ctx->sImix.shrink_to_fit();
    ctx->hydP.clear(); ctx->hydP.shrink_to_fit(); ctx->hydR.clear(); ctx->hydR.shrink_to_fit();
    fill_pingpong<double>(ctx, ctx->Pd, ctx->Pd_alt, ctx->Od);
    fill_pingpong<float>(ctx, ctx->Pf, ctx->Pf_alt, ctx->Of);
    int ctas = 0;
    e = mixed(ctx) ? prepare_fused<float>(ctx->Pf, &ctas) : prepare_fused<double>(ctx->Pd, &ctas);
    if (e != cudaSuccess) return cuda_check(ctx, e, "fused step set-up");
    for (int k = 0; k < 2; ++k) ctx->Od[k].ctas = ctx->Of[k].ctas = ctas;
    if (!mixed(ctx)) prepare_beside(ctx);
    // Default form.  Without gravity the fused form: its quiescent tiles (matter at rest
    // at zero pressure) only read and write their state, which on an impact grid is most of
    // it (4000 x 4000: mixed form 0.41 against 0.90 ms per step, FP64 1.26 against 7.16; a
    // 1600 x 1600 grid with a fifth of its vertices moving: 0.125 against 0.172, 1.02
    // against 1.47).  Under gravity no tile is quiescent (a loaded column is not at zero
    // pressure) and the phase kernels, which compute no cell twice, are faster (the
    // paper's layered grid: 0.054 against 0.087 ms, FP64 0.45 against 0.70).
    ctx->form = g.gravity == 0.0 ? SALEC_STEP_FUSED : SALEC_STEP_PHASES;
    ctx->parity = 0;
    ctx->rates_valid = false;
    ctx->finalized = true;
    return SALEC_OK;
}

constexpr int kGraphChunk = 16;

// Capture kGraphChunk steps on a private stream (a graph can then be launched into any
// stream, the legacy default stream included).  `launch(cs, k)` enqueues step k of the
// chunk.  nullptr, with no error left pending, when capture is not possible.
extern "C++" {
template <typename F>
static cudaGraphExec_t capture_chunk(F&& launch)
{
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int k = 0; k < kGraphChunk && e == cudaSuccess; ++k) e = launch(cs, k);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return x;
}
}  // extern "C++"

static bool capture_step_graph(salec_ctx* ctx)
{
    if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
    ctx->graph = capture_chunk([&](cudaStream_t cs, int) {
        return mixed(ctx) ? launch_step<float>(ctx->Pf, ctx->shape, cs, nullptr)
                          : launch_step<double>(ctx->Pd, ctx->shape, cs, nullptr);
    });
    if (!ctx->graph) return false;
    for (int k = 0; k < 6; ++k) ctx->graph_shape[k] = ctx->shape[k];
    return true;
}

// one fused step from the current copy; the next step reads the other one.  With the copy
// of tiles at rest switched off, the step's rest flags are cleared first: every tile then
// goes through the tile kernel.
static cudaError_t fused_step(salec_ctx* ctx, int parity, cudaStream_t s, cudaEvent_t* ev)
{
    if (!ctx->rest_copy) {
        const cudaError_t e = cudaMemsetAsync(ctx->base + ctx->L.rest[parity], 0, ctx->L.ntiles, s);
        if (e != cudaSuccess) return e;
    }
    if (beside(ctx))
        return launch_step_fused_beside(parity ? ctx->Pd_alt : ctx->Pd, ctx->Od[parity], ctx->rcopy[parity], s, ctx->s2,
                                        ctx->fork, ctx->join, ev);
    return mixed(ctx) ? launch_step_fused<float>(parity ? ctx->Pf_alt : ctx->Pf, ctx->Of[parity], s, ev)
                      : launch_step_fused<double>(parity ? ctx->Pd_alt : ctx->Pd, ctx->Od[parity], s, ev);
}

static bool same_shapes(const dim3* a, const dim3* b)
{
    for (int k = 0; k < 6; ++k)
        if (a[k].x != b[k].x || a[k].y != b[k].y) return false;
    return true;
}

// events per recorded step: one before the first kernel and one after each timed kernel
static int timed_kernels(const salec_ctx* ctx) { return ctx->form == SALEC_STEP_FUSED ? 2 : launches_per_step(); }

static salec_status step_fused(salec_ctx* ctx, int nsteps)
{
    if (nsteps == 0) return SALEC_OK;
    // the running Courant maximum must hold the current state's rates: a fused step leaves
    // them for the next one; anything else (set-up, host writes, phase or batched steps)
    // needs one pass over the state first, which also flags the tiles that the quiescent
    // path would return unchanged (the first step copies those whose neighbours are flagged)
    if (!ctx->rates_valid) {
        const Layout& L = ctx->L;
        cudaError_t e = canonical(ctx);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(ctx->base + L.scal + offsetof(DevScalars, maxbits), 0, sizeof(unsigned long long), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->base + L.rest[0], 0, L.work + 2 * sizeof(TileWork) - L.rest[0], ctx->stream);
        if (e == cudaSuccess && ctx->rest_copy) e = cudaMemsetAsync(ctx->base + L.rest[0], 1, L.ntiles, ctx->stream);
        unsigned char* rest0 = ctx->rest_copy ? at<unsigned char>(ctx, L.rest[0]) : nullptr;
        if (e == cudaSuccess) e = mixed(ctx) ? launch_courant_rates<float>(ctx->Pf, rest0, ctx->stream)
                                             : launch_courant_rates<double>(ctx->Pd, rest0, ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "Courant rates");
        ctx->rates_valid = true;
    }
    if (!ctx->timing && nsteps >= kGraphChunk && ctx->fgraph_ok) {
        const int p0 = ctx->parity;
        if (!ctx->fgraph[p0]) {
            ctx->fgraph[p0] = capture_chunk([&](cudaStream_t cs, int k) { return fused_step(ctx, (p0 + k) & 1, cs, nullptr); });
            if (!ctx->fgraph[p0]) ctx->fgraph_ok = false;
        }
        if (ctx->fgraph[p0]) {
            // a chunk has an even number of steps: it ends on the copy it started from
            for (; nsteps >= kGraphChunk; nsteps -= kGraphChunk) {
                const cudaError_t e = cudaGraphLaunch(ctx->fgraph[p0], ctx->stream);
                if (e != cudaSuccess) return cuda_check(ctx, e, "fused step graph launch");
            }
        }
    }
    for (int n = 0; n < nsteps; ++n) {
        cudaEvent_t* evp = nullptr;
        if (ctx->timing) {
            const size_t E = (size_t)events_per_step(ctx);
            while (ctx->ev_used + E > ctx->ev.size()) {
                cudaEvent_t e0;
                cudaError_t ce = cudaEventCreate(&e0);
                if (ce != cudaSuccess) return cuda_check(ctx, ce, "event create");
                ctx->ev.push_back(e0);
            }
            evp = ctx->ev.data() + ctx->ev_used;
            ctx->ev_used += E;
        }
        const cudaError_t e = fused_step(ctx, ctx->parity, ctx->stream, evp);
        if (e != cudaSuccess) return cuda_check(ctx, e, "fused step launch");
        ctx->parity ^= 1;
    }
    return SALEC_OK;
}

salec_status salec_step(salec_ctx* ctx, int nsteps)
{
    HostRange range("salec_step");
    if (!ctx || nsteps < 0) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "step before finalize");
    if (ctx->form == SALEC_STEP_FUSED) return step_fused(ctx, nsteps);
    cudaError_t ce = canonical(ctx);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "canonical copy");
    if (nsteps > 0) ctx->rates_valid = false;
    // whole chunks as graph replays (the kernel arguments are fixed after finalize; the
    // graph is captured again when the block shapes change)
    if (!ctx->timing && nsteps >= kGraphChunk && ctx->graph_ok) {
        if (ctx->graph && !same_shapes(ctx->graph_shape, ctx->shape)) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
        if (!ctx->graph) ctx->graph_ok = capture_step_graph(ctx);
        if (ctx->graph) {
            for (; nsteps >= kGraphChunk; nsteps -= kGraphChunk) {
                const cudaError_t e = cudaGraphLaunch(ctx->graph, ctx->stream);
                if (e != cudaSuccess) return cuda_check(ctx, e, "step graph launch");
            }
        }
    }
    const int K = launches_per_step() + 1;
    for (int n = 0; n < nsteps; ++n) {
        cudaEvent_t* evp = nullptr;
        if (ctx->timing) {
            while (ctx->ev_used + K > ctx->ev.size()) {
                cudaEvent_t e0;
                cudaError_t ce = cudaEventCreate(&e0);
                if (ce != cudaSuccess) return cuda_check(ctx, ce, "event create");
                ctx->ev.push_back(e0);
            }
            evp = ctx->ev.data() + ctx->ev_used;
            ctx->ev_used += K;
        }
        cudaError_t e = mixed(ctx) ? launch_step<float>(ctx->Pf, ctx->shape, ctx->stream, evp)
                                   : launch_step<double>(ctx->Pd, ctx->shape, ctx->stream, evp);
        if (e != cudaSuccess) return cuda_check(ctx, e, "step launch");
    }
    return SALEC_OK;
}

salec_status salec_set_step_form(salec_ctx* ctx, int form)
{
    if (!ctx || (form != SALEC_STEP_PHASES && form != SALEC_STEP_FUSED)) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "set_step_form before finalize");
    if (form == ctx->form) return SALEC_OK;
    const cudaError_t e = canonical(ctx);
    if (e != cudaSuccess) return cuda_check(ctx, e, "canonical copy");
    ctx->form = form;
    ctx->rates_valid = false;
    ctx->ev_used = 0;
    return SALEC_OK;
}

int salec_get_step_form(const salec_ctx* ctx) { return ctx ? ctx->form : -1; }

salec_status salec_set_rest_copy(salec_ctx* ctx, int mode)
{
    if (!ctx || mode < 0 || mode > 2) return SALEC_EINVAL;
    const bool on = mode != 0, by = mode == 2;
    if (on == ctx->rest_copy && by == ctx->copy_beside) return SALEC_OK;
    ctx->rest_copy = on;
    ctx->copy_beside = by;
    ctx->ev_used = 0;
    for (int k = 0; k < 2; ++k)
        if (ctx->fgraph[k]) { cudaGraphExecDestroy(ctx->fgraph[k]); ctx->fgraph[k] = nullptr; }
    return SALEC_OK;
}

salec_status salec_set_kernel_timing(salec_ctx* ctx, int on)
{
    if (!ctx) return SALEC_EINVAL;
    ctx->timing = on != 0;
    ctx->ev_used = 0;
    return SALEC_OK;
}

salec_status salec_kernel_times(salec_ctx* ctx, double* avg_ms, int n, int* steps)
{
    if (!ctx || !avg_ms || !steps) return SALEC_EINVAL;
    const int K = timed_kernels(ctx);
    if (n < K) return SALEC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kernel times");
    const size_t E = (size_t)events_per_step(ctx);
    const size_t ns = ctx->ev_used / E;
    for (int k = 0; k < n; ++k) avg_ms[k] = 0.0;
    for (size_t s = 0; s < ns; ++s)
        for (int k = 0; k < K; ++k) {
            float ms = 0.0f;
            int a = 0, b = 0;
            kernel_events(ctx, k, &a, &b);
            e = cudaEventElapsedTime(&ms, ctx->ev[s * E + a], ctx->ev[s * E + b]);
            if (e != cudaSuccess) return cuda_check(ctx, e, "event elapsed");
            avg_ms[k] += ms;
        }
    for (int k = 0; k < K; ++k) avg_ms[k] = ns ? avg_ms[k] / (double)ns : 0.0;
    *steps = (int)ns;
    ctx->ev_used = 0;
    return SALEC_OK;
}

const char* salec_kernel_name(int k)
{
    return kernel_name(k);
}

const char* salec_step_kernel_name(const salec_ctx* ctx, int k)
{
    if (ctx && ctx->form == SALEC_STEP_FUSED)
        return k == 0 ? (beside(ctx) ? "k_rest_copy" : "k_rest_tiles") : k == 1 ? "k_step_fused" : "";
    return kernel_name(k);
}

salec_status salec_get_scalars(salec_ctx* ctx, double out[8])
{
    if (!ctx || !out) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "scalars before finalize");
    DevScalars s;
    cudaError_t e = cudaMemcpyAsync(&s, ctx->base + ctx->L.scal, sizeof(s), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "read scalars");
    out[0] = s.t; out[1] = s.dt; out[2] = (double)s.nstep; out[3] = (double)s.status;
    out[4] = s.mass_out; out[5] = s.mass_discarded; out[6] = s.mass_pml; out[7] = s.zmom_out;
    if (s.status != 0) return fail(ctx, SALEC_EUNSTABLE, "device status %d", s.status);
    return SALEC_OK;
}

salec_status salec_set_time(salec_ctx* ctx, double t, double dt_prev)
{
    if (!ctx) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "set_time before finalize");
    DevScalars s;
    cudaError_t e = cudaMemcpyAsync(&s, ctx->base + ctx->L.scal, sizeof(s), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    s.t = t;
    s.dt_prev = dt_prev;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->base + ctx->L.scal, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "set_time");
}

// Where a field lives: a device array of `stride` doubles per element, component `comp`,
// over the whole grid (strip == 0) or over a PML strip (1 bottom cells, 2 right cells,
// 3 bottom vertices, 4 right vertices).
struct FieldLoc { size_t off; int stride, comp, strip; bool vertex; size_t es; };

static bool locate(const salec_ctx* ctx, int field, FieldLoc& F)
{
    const Layout& L = ctx->L;
    F.strip = 0; F.vertex = false; F.stride = 1; F.comp = 0; F.es = L.es;
    if (field >= SALEC_F_VOLFRAC0 && field <= SALEC_F_VOLFRAC2) {
        if (field - SALEC_F_VOLFRAC0 >= ctx->g.nmat) return false;
        F.off = L.fr[field - SALEC_F_VOLFRAC0]; F.stride = 2; F.comp = 0; return true;
    }
    if (field >= SALEC_F_DENS0 && field <= SALEC_F_DENS2) {
        if (field - SALEC_F_DENS0 >= ctx->g.nmat) return false;
        F.off = L.fr[field - SALEC_F_DENS0]; F.stride = 2; F.comp = 1; return true;
    }
    switch (field) {
    case SALEC_F_IE: F.off = L.I; F.es = sizeof(double); return true;
    case SALEC_F_SRR: F.off = L.s01; F.stride = 2; F.comp = 0; return true;
    case SALEC_F_SZZ: F.off = L.s01; F.stride = 2; F.comp = 1; return true;
    case SALEC_F_SRZ: F.off = L.s2d; F.stride = 2; F.comp = 0; return true;
    case SALEC_F_DAMAGE: F.off = L.s2d; F.stride = 2; F.comp = 1; return true;
    case SALEC_F_PMAX: F.off = L.pmax; return true;
    case SALEC_F_VR: F.off = L.v; F.stride = 2; F.comp = 0; F.vertex = true; return true;
    case SALEC_F_VZ: F.off = L.v; F.stride = 2; F.comp = 1; F.vertex = true; return true;
    case SALEC_F_PHI1_B: F.off = L.pb_c; F.stride = 2; F.comp = 0; F.strip = 1; return true;
    case SALEC_F_PHI3_B: F.off = L.pb_c; F.stride = 2; F.comp = 1; F.strip = 1; return true;
    case SALEC_F_PSI2_B: F.off = L.pb_psi2; F.strip = 1; return true;
    case SALEC_F_PHI1_R: F.off = L.pr_c; F.stride = 2; F.comp = 0; F.strip = 2; return true;
    case SALEC_F_PHI3_R: F.off = L.pr_c; F.stride = 2; F.comp = 1; F.strip = 2; return true;
    case SALEC_F_PSI2_R: F.off = L.pr_psi2; F.strip = 2; return true;
    default: break;
    }
    if (field >= SALEC_F_PHI2R_B && field <= SALEC_F_PSI1Z_R) {
        const int k = field - SALEC_F_PHI2R_B;
        F.vertex = true; F.stride = 4; F.comp = k % 4;
        F.strip = k < 4 ? 3 : 4;
        F.off = k < 4 ? L.pb_v : L.pr_v;
        return true;
    }
    return false;
}

// number of elements of the device array behind a location, and the map from a
// full-grid index to it (-1 outside the strip)
static size_t loc_count(const salec_ctx* ctx, const FieldLoc& F)
{
    const size_t nr = ctx->g.nr, nz = ctx->g.nz, pr = ctx->g.pml_right, pb = ctx->g.pml_bottom;
    switch (F.strip) {
    case 1: return nr * pb;
    case 2: return pr * nz;
    case 3: return (nr + 1) * pb;
    case 4: return pr * (nz + 1);
    default: return F.vertex ? (nr + 1) * (nz + 1) : nr * nz;
    }
}
static long strip_index(const salec_ctx* ctx, const FieldLoc& F, int i, int j)
{
    const int nr = ctx->g.nr, pr = ctx->g.pml_right, pb = ctx->g.pml_bottom;
    switch (F.strip) {
    case 1: return j < pb ? (long)j * nr + i : -1;
    case 2: return i >= nr - pr ? (long)j * pr + (i - (nr - pr)) : -1;
    case 3: return j < pb ? (long)j * (nr + 1) + i : -1;
    case 4: return i > nr - pr ? (long)j * pr + (i - (nr - pr + 1)) : -1;
    default: return F.vertex ? (long)j * (nr + 1) + i : (long)j * nr + i;
    }
}

// the current fields in the first copy before an accessor reads or writes them; a write also
// invalidates the running Courant maximum
static salec_status current_fields(salec_ctx* ctx, bool write)
{
    const cudaError_t e = canonical(ctx);
    if (e != cudaSuccess) return cuda_check(ctx, e, "canonical copy");
    if (write) ctx->rates_valid = false;
    return SALEC_OK;
}

salec_status salec_get_field(salec_ctx* ctx, int field, double* host_out, size_t n)
{
    if (!ctx || !host_out) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "get_field before finalize");
    if (salec_status st = current_fields(ctx, false)) return st;
    const int nr = ctx->g.nr, nz = ctx->g.nz;
    const size_t nc = (size_t)nr * nz;
    if (field == SALEC_F_PRESSURE) {
        if (n != nc) return fail(ctx, SALEC_EINVAL, "pressure needs n = nr*nz");
        double* tmp = at<double>(ctx, ctx->L.tmp);
        cudaError_t e = mixed(ctx) ? launch_pressure<float>(ctx->Pf, tmp, ctx->stream)
                                   : launch_pressure<double>(ctx->Pd, tmp, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        return cuda_check(ctx, e, "get pressure");
    }
    FieldLoc F;
    if (!locate(ctx, field, F)) return fail(ctx, SALEC_EINVAL, "unknown field %d", field);
    const size_t want = F.vertex ? (size_t)(nr + 1) * (nz + 1) : nc;
    if (n != want) return fail(ctx, SALEC_EINVAL, "field %d needs n = %zu", field, want);
    const size_t cnt = loc_count(ctx, F);
    std::vector<double> buf(cnt * F.stride + 1);
    std::vector<float> fbuf(F.es == sizeof(float) ? cnt * F.stride + 1 : 0);
    void* dst = F.es == sizeof(float) ? (void*)fbuf.data() : (void*)buf.data();
    cudaError_t e = cudaSuccess;
    if (cnt) e = cudaMemcpyAsync(dst, ctx->base + F.off, cnt * F.stride * F.es, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "get field");
    if (F.es == sizeof(float))
        for (size_t k = 0; k < cnt * F.stride; ++k) buf[k] = (double)fbuf[k];
    const int ni = F.vertex ? nr + 1 : nr, nj = F.vertex ? nz + 1 : nz;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const long k = strip_index(ctx, F, i, j);
            host_out[(size_t)j * ni + i] = k < 0 ? 0.0 : buf[(size_t)k * F.stride + F.comp];
        }
    return SALEC_OK;
}

salec_status salec_set_field(salec_ctx* ctx, int field, const double* host_in, size_t n)
{
    if (!ctx || !host_in) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "set_field before finalize");
    if (field == SALEC_F_PRESSURE) return fail(ctx, SALEC_EINVAL, "pressure is read-only");
    if (salec_status st = current_fields(ctx, true)) return st;
    const int nr = ctx->g.nr, nz = ctx->g.nz;
    FieldLoc F;
    if (!locate(ctx, field, F)) return fail(ctx, SALEC_EINVAL, "unknown field %d", field);
    const size_t want = F.vertex ? (size_t)(nr + 1) * (nz + 1) : (size_t)nr * nz;
    if (n != want) return fail(ctx, SALEC_EINVAL, "field %d needs n = %zu", field, want);
    const size_t cnt = loc_count(ctx, F);
    if (!cnt) return SALEC_OK;
    std::vector<double> buf(cnt * F.stride);
    std::vector<float> fbuf(F.es == sizeof(float) ? cnt * F.stride : 0);
    void* raw = F.es == sizeof(float) ? (void*)fbuf.data() : (void*)buf.data();
    cudaError_t e = cudaMemcpyAsync(raw, ctx->base + F.off, cnt * F.stride * F.es, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "set field (read)");
    if (F.es == sizeof(float))
        for (size_t k = 0; k < cnt * F.stride; ++k) buf[k] = (double)fbuf[k];
    const int ni = F.vertex ? nr + 1 : nr, nj = F.vertex ? nz + 1 : nz;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const long k = strip_index(ctx, F, i, j);
            if (k >= 0) buf[(size_t)k * F.stride + F.comp] = host_in[(size_t)j * ni + i];
        }
    if (F.es == sizeof(float))
        for (size_t k = 0; k < cnt * F.stride; ++k) fbuf[k] = (float)buf[k];
    e = cudaMemcpyAsync(ctx->base + F.off, raw, cnt * F.stride * F.es, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "set field (write)");
}

salec_status salec_crater_profile(salec_ctx* ctx, double z_surface, int npts, double* depth_profile, double* heights,
                                  double* depth, double* diameter)
{
    if (!ctx || !depth || !diameter || npts < 0 || (npts > 0 && !depth_profile)) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "crater_profile before finalize");
    if (salec_status st = current_fields(ctx, false)) return st;
    const int nr = ctx->g.nr;
    const std::vector<double>& rc = ctx->rc;
    std::vector<double> h(nr);
    double* tmp = at<double>(ctx, ctx->L.tmp);
    cudaError_t e = mixed(ctx) ? launch_column_heights<float>(ctx->Pf, tmp, ctx->stream)
                               : launch_column_heights<double>(ctx->Pd, tmp, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), tmp, nr * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "crater profile");
    // depth on the axis; deepest column; first up-crossing of z_surface beyond it
    int kmin = 0;
    for (int i = 1; i < nr; ++i) if (z_surface - h[i] > z_surface - h[kmin]) kmin = i;
    double D = 0.0;
    if (z_surface - h[kmin] > 0.0) {
        D = 2.0 * rc[nr - 1];
        for (int i = kmin; i + 1 < nr; ++i)
            if (h[i] < z_surface && z_surface <= h[i + 1]) {
                D = 2.0 * (rc[i] + (z_surface - h[i]) / (h[i + 1] - h[i]) * (rc[i + 1] - rc[i]));
                break;
            }
    }
    if (npts > 0) {
        // the depth profile sampled at r_k = (k + 1/2) r_ext / npts, r_ext the inner edge
        // of the right strip, linear between column centres
        const double rext = ctx->rR[nr - ctx->g.pml_right];
        int i0 = 0;
        for (int k = 0; k < npts; ++k) {
            const double r = ((double)k + 0.5) * rext / npts;
            double val;
            if (r <= rc[0]) val = z_surface - h[0];
            else if (r >= rc[nr - 1]) val = z_surface - h[nr - 1];
            else {
                while (rc[i0 + 1] < r) ++i0;
                const double w = (r - rc[i0]) / (rc[i0 + 1] - rc[i0]);
                val = (1.0 - w) * (z_surface - h[i0]) + w * (z_surface - h[i0 + 1]);
            }
            depth_profile[k] = val;
        }
    }
    if (heights) memcpy(heights, h.data(), nr * sizeof(double));
    *depth = z_surface - h[0];
    *diameter = D;
    return SALEC_OK;
}

salec_status salec_conservation(salec_ctx* ctx, double out[4])
{
    if (!ctx || !out) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "conservation before finalize");
    if (salec_status st = current_fields(ctx, false)) return st;
    double* part = at<double>(ctx, ctx->L.partial);
    int nb = 0;
    cudaError_t e = mixed(ctx) ? launch_conservation<float>(ctx->Pf, part, &nb, ctx->stream)
                               : launch_conservation<double>(ctx->Pd, part, &nb, ctx->stream);
    std::vector<double> h((size_t)4 * nb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "conservation");
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 4; ++k) s[k] += h[(size_t)4 * b + k];
    for (int k = 0; k < 4; ++k) out[k] = s[k];
    return SALEC_OK;
}

salec_status salec_checkpoint_bytes(salec_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return SALEC_EINVAL;
    *bytes = ctx->L.persist_end;
    return SALEC_OK;
}

salec_status salec_get_state(salec_ctx* ctx, void* host, size_t bytes)
{
    if (!ctx || !host) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "get_state before finalize");
    if (bytes != ctx->L.persist_end) return fail(ctx, SALEC_EINVAL, "checkpoint needs %zu bytes", ctx->L.persist_end);
    if (salec_status st = current_fields(ctx, false)) return st;
    cudaError_t e = cudaMemcpyAsync(host, ctx->base, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "get_state");
}

salec_status salec_set_state(salec_ctx* ctx, const void* host, size_t bytes)
{
    if (!ctx || !host) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "set_state before finalize");
    if (bytes != ctx->L.persist_end) return fail(ctx, SALEC_EINVAL, "checkpoint needs %zu bytes", ctx->L.persist_end);
    if (salec_status st = current_fields(ctx, true)) return st;
    cudaError_t e = cudaMemcpyAsync(ctx->base, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "set_state");
}

salec_status salec_state_changed(salec_ctx* ctx)
{
    if (!ctx) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "state_changed before finalize");
    ctx->parity = 0;
    ctx->rates_valid = false;
    return SALEC_OK;
}

salec_status salec_set_end_time(salec_ctx* ctx, double t_end)
{
    if (!ctx) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "set_end_time before finalize");
    DevScalars* d = at<DevScalars>(ctx, ctx->L.scal);
    cudaError_t e = cudaMemcpyAsync(&d->t_end, &t_end, sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_check(ctx, e, "set_end_time");
}

static bool shape_ok(unsigned x, unsigned y)
{
    return x >= 32 && x % 32 == 0 && y >= 1 && x * y <= (unsigned)kMaxThreads && x * y >= 128;
}

salec_status salec_set_block_shapes(salec_ctx* ctx, const int* shapes)
{
    if (!ctx || !shapes) return SALEC_EINVAL;
    for (int k = 0; k < 6; ++k)
        if (!shape_ok((unsigned)shapes[2 * k], (unsigned)shapes[2 * k + 1]))
            return fail(ctx, SALEC_EINVAL, "block shape %d x %d not allowed", shapes[2 * k], shapes[2 * k + 1]);
    for (int k = 0; k < 6; ++k) ctx->shape[k] = dim3(shapes[2 * k], shapes[2 * k + 1]);
    return SALEC_OK;
}

salec_status salec_get_block_shapes(const salec_ctx* ctx, int* shapes)
{
    if (!ctx || !shapes) return SALEC_EINVAL;
    for (int k = 0; k < 6; ++k) { shapes[2 * k] = (int)ctx->shape[k].x; shapes[2 * k + 1] = (int)ctx->shape[k].y; }
    return SALEC_OK;
}

// Autotuner: every candidate block shape runs `trial_steps` real steps of this simulation
// (after one untimed step) with per-kernel events; each kernel keeps its fastest shape.
// The state after the call is the state after all those steps: the block shape does not
// change any field (only the summation order of the diagnostic tallies).
salec_status salec_autotune(salec_ctx* ctx, int trial_steps, int* shapes_out)
{
    HostRange range("salec_autotune");
    if (!ctx || trial_steps < 1) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "autotune before finalize");
    // the block shapes are those of the phase kernels: tune them in the phase form
    const int form = ctx->form;
    if (salec_status st = salec_set_step_form(ctx, SALEC_STEP_PHASES)) return st;
    const int K = launches_per_step();
    double best[6];
    dim3 pick[6];
    for (int k = 0; k < K; ++k) { best[k] = 1e300; pick[k] = ctx->shape[k]; }
    const bool was_timing = ctx->timing;
    for (int c = 0; c < kNumShapes; ++c) {
        for (int k = 0; k < K; ++k) ctx->shape[k] = kShapes[c];
        ctx->timing = false;
        salec_status st = salec_step(ctx, 1);
        if (st != SALEC_OK) return st;
        salec_set_kernel_timing(ctx, 1);
        st = salec_step(ctx, trial_steps);
        if (st != SALEC_OK) return st;
        double ms[8];
        int ns = 0;
        st = salec_kernel_times(ctx, ms, 8, &ns);
        if (st != SALEC_OK) return st;
        for (int k = 0; k < K; ++k)
            if (ms[k] < best[k]) { best[k] = ms[k]; pick[k] = kShapes[c]; }
    }
    for (int k = 0; k < K; ++k) ctx->shape[k] = pick[k];
    ctx->timing = was_timing;
    ctx->ev_used = 0;
    if (shapes_out) salec_get_block_shapes(ctx, shapes_out);
    return salec_set_step_form(ctx, form);
}

// ---------------------------------------------------------------------------------
// Batches: many independent runs advanced by one set of launches per step.
// ---------------------------------------------------------------------------------
struct salec_batch {
    std::vector<salec_ctx*> runs;
    int precision = 0, nmat = 0;
    bool strength = false;
    bool uniform = false;       // every run on a uniform grid
    cudaStream_t stream = nullptr;
    char* dev = nullptr;
    size_t bytes = 0;
    size_t off_params = 0, off_poll = 0, off_work[6] = {0, 0, 0, 0, 0, 0};
    int ntiles[6] = {0, 0, 0, 0, 0, 0};
    std::vector<char> retired;      // runs left out of the work lists (reached their end time)
    dim3 shape[6];
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::string err;
    // persistent mode (salec_batch_set_persistent): one cooperative launch per chunk
    bool persistent = false;
    int pctas = 0;                  // resident blocks of the persistent kernel
    bool pgraph = true;             // its launch is captured in the chunk graph (false: capture refused)
    size_t off_sync = 0;            // its grid barrier
    bool expire_next = false;       // salec_batch_expire_next_barrier
};

static salec_status bfail(salec_batch* b, salec_status st, const char* msg)
{
    if (b) b->err = msg;
    return st;
}

// bytes of the batch buffer: run parameter blocks, a poll area, and for each kernel the
// largest work list any allowed block shape needs
static size_t batch_layout(salec_ctx* const* runs, int n, salec_batch* b)
{
    size_t cur = 0;
    const size_t psize = runs[0]->precision == SALEC_FP32MIX ? sizeof(ParamsT<float>) : sizeof(ParamsT<double>);
    const size_t op = take(cur, psize * (size_t)n);
    const size_t opoll = take(cur, sizeof(double) * 5 * (size_t)n);
    const size_t osync = take(cur, sizeof(GridSync));
    size_t ow[6];
    for (int k = 0; k < 6; ++k) {
        size_t cap = 0;
        for (int r = 0; r < n; ++r) {
            size_t mx = 0;
            for (int c = 0; c < kNumShapes; ++c) {
                const size_t t = (size_t)tiles_of(runs[r]->g.nr, runs[r]->g.nz, k, kShapes[c]);
                mx = t > mx ? t : mx;
            }
            cap += mx;
        }
        ow[k] = take(cur, cap * sizeof(BatchTile));
    }
    if (b) {
        b->off_params = op;
        b->off_poll = opoll;
        b->off_sync = osync;
        for (int k = 0; k < 6; ++k) b->off_work[k] = ow[k];
    }
    return cur;
}

static salec_status batch_check(salec_ctx* const* runs, int n)
{
    if (!runs || n < 1) return SALEC_EINVAL;
    for (int r = 0; r < n; ++r) {
        if (!runs[r] || !runs[r]->finalized) return SALEC_EORDER;
        if (runs[r]->precision != runs[0]->precision || runs[r]->g.nmat != runs[0]->g.nmat) return SALEC_EINVAL;
        const int s0 = runs[0]->Pd.any_strength, sr = runs[r]->Pd.any_strength;
        if (s0 != sr) return SALEC_EINVAL;
        if (runs[r]->g.nr + 1 > 0xffff * 32 || runs[r]->g.nz + 1 > 0xffff) return SALEC_EINVAL;
    }
    return SALEC_OK;
}

salec_status salec_batch_bytes(salec_ctx* const* runs, int nruns, size_t* bytes)
{
    const salec_status st = batch_check(runs, nruns);
    if (st != SALEC_OK || !bytes) return st != SALEC_OK ? st : SALEC_EINVAL;
    *bytes = batch_layout(runs, nruns, nullptr);
    return SALEC_OK;
}

static salec_status batch_build_work(salec_batch* b)
{
    b->retired.resize(b->runs.size(), 0);
    for (int k = 0; k < 6; ++k) {
        std::vector<BatchTile> w;
        for (int r = 0; r < (int)b->runs.size(); ++r) {
            if (b->retired[r]) continue;
            const salec_grid& g = b->runs[r]->g;
            const int ni = kernel_on_vertices(k) ? g.nr + 1 : g.nr, nj = kernel_on_vertices(k) ? g.nz + 1 : g.nz;
            const int gx = (ni + (int)b->shape[k].x - 1) / (int)b->shape[k].x;
            const int gy = (nj + (int)b->shape[k].y - 1) / (int)b->shape[k].y;
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) w.push_back(BatchTile{r, bx, by, gx | (gy << 16)});
        }
        b->ntiles[k] = (int)w.size();
        cudaError_t e = cudaMemcpyAsync(b->dev + b->off_work[k], w.data(), w.size() * sizeof(BatchTile),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
    }
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
    return SALEC_OK;
}

salec_status salec_batch_create(salec_ctx* const* runs, int nruns, void* dev_buf, size_t bytes, void* stream,
                                salec_batch** out)
{
    salec_status st = batch_check(runs, nruns);
    if (st != SALEC_OK || !out) return st != SALEC_OK ? st : SALEC_EINVAL;
    for (int r = 0; r < nruns; ++r)
        if ((st = current_fields(runs[r], true)) != SALEC_OK) return st;
    salec_batch* b = new salec_batch();
    const size_t need = batch_layout(runs, nruns, b);
    if (!dev_buf || bytes < need || ((uintptr_t)dev_buf % kAlign) != 0) { delete b; return SALEC_ENOMEM; }
    b->runs.assign(runs, runs + nruns);
    b->precision = runs[0]->precision;
    b->nmat = runs[0]->g.nmat;
    b->strength = runs[0]->Pd.any_strength != 0;
    b->uniform = true;
    for (int k = 0; k < nruns; ++k) b->uniform = b->uniform && runs[k]->uniform;
    b->stream = (cudaStream_t)stream;
    b->dev = (char*)dev_buf;
    b->bytes = bytes;
    for (int k = 0; k < 6; ++k) b->shape[k] = kDefaultShape;
    // run parameter blocks
    cudaError_t e = cudaSuccess;
    if (b->precision == SALEC_FP32MIX) {
        std::vector<ParamsT<float>> P(nruns);
        for (int r = 0; r < nruns; ++r) P[r] = runs[r]->Pf;
        e = cudaMemcpyAsync(b->dev + b->off_params, P.data(), P.size() * sizeof(P[0]), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    } else {
        std::vector<ParamsT<double>> P(nruns);
        for (int r = 0; r < nruns; ++r) P[r] = runs[r]->Pd;
        e = cudaMemcpyAsync(b->dev + b->off_params, P.data(), P.size() * sizeof(P[0]), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) { delete b; return SALEC_ECUDA; }
    st = batch_build_work(b);
    if (st != SALEC_OK) { delete b; return st; }
    *out = b;
    return SALEC_OK;
}

static cudaError_t batch_launch(salec_batch* b, cudaEvent_t* ev)
{
    const BatchTile* work[6];
    for (int k = 0; k < 6; ++k) work[k] = reinterpret_cast<const BatchTile*>(b->dev + b->off_work[k]);
    if (b->precision == SALEC_FP32MIX)
        return launch_batch_step<float>(reinterpret_cast<const ParamsT<float>*>(b->dev + b->off_params), (int)b->runs.size(), b->nmat,
                                        b->strength, b->uniform, work, b->ntiles, b->shape, b->stream, ev);
    return launch_batch_step<double>(reinterpret_cast<const ParamsT<double>*>(b->dev + b->off_params), (int)b->runs.size(), b->nmat,
                                     b->strength, b->uniform, work, b->ntiles, b->shape, b->stream, ev);
}

// Persistent mode: `steps` steps of every run in one cooperative launch (the cell work list
// of kernel 0 and the vertex list of kernel 1; every kernel has the same block shape).
static cudaError_t batch_launch_persistent(salec_batch* b, int steps, bool expire = false)
{
    const BatchTile* cells = reinterpret_cast<const BatchTile*>(b->dev + b->off_work[0]);
    const BatchTile* verts = reinterpret_cast<const BatchTile*>(b->dev + b->off_work[1]);
    GridSync* gs = reinterpret_cast<GridSync*>(b->dev + b->off_sync);
    const int n = (int)b->runs.size();
    if (b->precision == SALEC_FP32MIX)
        return launch_batch_persistent<float>(reinterpret_cast<const ParamsT<float>*>(b->dev + b->off_params), n, b->nmat,
                                              b->strength, b->uniform, cells, b->ntiles[0], verts, b->ntiles[1], b->shape[0],
                                              b->pctas, steps, gs, expire, b->stream);
    return launch_batch_persistent<double>(reinterpret_cast<const ParamsT<double>*>(b->dev + b->off_params), n, b->nmat,
                                           b->strength, b->uniform, cells, b->ntiles[0], verts, b->ntiles[1], b->shape[0],
                                           b->pctas, steps, gs, expire, b->stream);
}

// the resident grid of the persistent kernel for the current block shape
static salec_status batch_prepare_persistent(salec_batch* b)
{
    const cudaError_t e = b->precision == SALEC_FP32MIX
                              ? prepare_batch_persistent<float>(b->nmat, b->strength, b->uniform, b->shape[0], &b->pctas)
                              : prepare_batch_persistent<double>(b->nmat, b->strength, b->uniform, b->shape[0], &b->pctas);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
    }
    return SALEC_OK;
}

static salec_status batch_restore_retired(salec_batch* b);

// a run stepped alone in the fused form since the last batched step has its fields in the
// second copy: bring them back (the batch's kernels work in place on the first)
static salec_status batch_fields(salec_batch* b)
{
    for (salec_ctx* r : b->runs)
        if (salec_status st = current_fields(r, true)) return bfail(b, st, r->err.c_str());
    return SALEC_OK;
}

salec_status salec_batch_step(salec_batch* b, int nsteps)
{
    HostRange range("salec_batch_step");
    if (!b || nsteps < 0) return SALEC_EINVAL;
    salec_status st0 = batch_fields(b);
    if (st0 == SALEC_OK) st0 = batch_restore_retired(b);
    if (st0 != SALEC_OK) return st0;
    if (b->persistent) {
        // one launch for the n steps; with timing on, an event before and one after it
        if (nsteps == 0) return SALEC_OK;
        cudaEvent_t* evp = nullptr;
        if (b->timing) {
            while (b->ev_used + 2 > b->ev.size()) {
                cudaEvent_t e0;
                if (cudaEventCreate(&e0) != cudaSuccess) return bfail(b, SALEC_ECUDA, "event create");
                b->ev.push_back(e0);
            }
            evp = b->ev.data() + b->ev_used;
            b->ev_used += 2;
            cudaEventRecord(evp[0], b->stream);
        }
        const cudaError_t e = batch_launch_persistent(b, nsteps, b->expire_next);
        b->expire_next = false;
        if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
        if (evp) cudaEventRecord(evp[1], b->stream);
        return SALEC_OK;
    }
    const int K = launches_per_step() + 1;
    for (int n = 0; n < nsteps; ++n) {
        cudaEvent_t* evp = nullptr;
        if (b->timing) {
            while (b->ev_used + K > b->ev.size()) {
                cudaEvent_t e0;
                if (cudaEventCreate(&e0) != cudaSuccess) return bfail(b, SALEC_ECUDA, "event create");
                b->ev.push_back(e0);
            }
            evp = b->ev.data() + b->ev_used;
            b->ev_used += K;
        }
        const cudaError_t e = batch_launch(b, evp);
        if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
    }
    return SALEC_OK;
}

// Scalars of every run: out[5 r + (0 t, 1 dt, 2 steps, 3 status, 4 t_end)] (synchronises).
salec_status salec_batch_poll(salec_batch* b, double* out)
{
    if (!b || !out) return SALEC_EINVAL;
    const int n = (int)b->runs.size();
    double* d = reinterpret_cast<double*>(b->dev + b->off_poll);
    cudaError_t e = b->precision == SALEC_FP32MIX
                        ? launch_batch_poll<float>(reinterpret_cast<const ParamsT<float>*>(b->dev + b->off_params), n, d, b->stream)
                        : launch_batch_poll<double>(reinterpret_cast<const ParamsT<double>*>(b->dev + b->off_params), n, d, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, b->stream);
    GridSync gs = {0, 0, 0, 0};
    if (e == cudaSuccess && b->persistent)
        e = cudaMemcpyAsync(&gs, b->dev + b->off_sync, sizeof(gs), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
    if (gs.err) {
        char msg[160];
        snprintf(msg, sizeof msg, "persistent batch: a grid-barrier wait ran out (step %d of the launch, barrier %d)",
                 (gs.where - 1) / 8, (gs.where - 1) % 8);
        return bfail(b, SALEC_ETIMEOUT, msg);
    }
    return SALEC_OK;
}

// Capture `chunk` batched steps as a CUDA graph on the batch stream.
static salec_status batch_capture(salec_batch* b, int chunk)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // do not leave the error for a later, unrelated check
        return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
    }
    if (b->persistent)
        e = batch_launch_persistent(b, chunk);
    else
        for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = batch_launch(b, nullptr);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return bfail(b, SALEC_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(b, SALEC_ECUDA, cudaGetErrorString(e)); }
    b->graph_steps = chunk;
    return SALEC_OK;
}

// A run left out of the work lists by an earlier salec_batch_run comes back if it is no
// longer finished (its end time was moved since); one poll decides.
static salec_status batch_restore_retired(salec_batch* b)
{
    bool any = false;
    for (char r : b->retired) any = any || r;
    if (!any) return SALEC_OK;
    const int n = (int)b->runs.size();
    std::vector<double> poll((size_t)5 * n);
    const salec_status st = salec_batch_poll(b, poll.data());
    if (st != SALEC_OK) return st;
    bool back = false;
    for (int r = 0; r < n; ++r)
        if (b->retired[r] && poll[5 * r] < poll[5 * r + 4] && poll[5 * r + 3] == 0.0) {
            b->retired[r] = 0;
            back = true;
        }
    return back ? batch_build_work(b) : SALEC_OK;
}

// Advance every run until it reaches its end time (salec_set_end_time) or fails (status
// not 0: it then stops where it failed), in CUDA-graph
// replays of `chunk` steps (the graph is captured once per block-shape set, chunk size and
// set of runs), polling completion after each replay; at most max_steps steps.  A run that
// is done does nothing in later steps (its blocks return at once); once done runs hold an
// eighth of the blocks they are left out of the work lists and the graph is captured again.
salec_status salec_batch_run(salec_batch* b, int chunk, long max_steps, long* steps_done, int* runs_done)
{
    HostRange range("salec_batch_run");
    if (!b || chunk < 1 || max_steps < 0) return SALEC_EINVAL;
    const int n = (int)b->runs.size();
    if (b->stream == nullptr || b->stream == cudaStreamLegacy || b->stream == cudaStreamPerThread)
        return bfail(b, SALEC_EINVAL, "batch_run captures a CUDA graph and needs a created stream, "
                                      "not a default stream");
    salec_status st0 = batch_fields(b);
    if (st0 == SALEC_OK) st0 = batch_restore_retired(b);
    if (st0 != SALEC_OK) return st0;
    if (b->graph && b->graph_steps != chunk) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    std::vector<double> poll((size_t)5 * n);
    long done_steps = 0;
    int done = 0;
    while (done_steps < max_steps) {
        if (b->persistent && !b->pgraph) {
            // the cooperative launch could not be captured: launch it directly
            const cudaError_t e = batch_launch_persistent(b, chunk);
            if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
        } else {
            if (!b->graph) {
                const salec_status st = batch_capture(b, chunk);
                if (st != SALEC_OK && b->persistent) {
                    b->pgraph = false;
                    continue;
                }
                if (st != SALEC_OK) return st;
            }
            const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bfail(b, SALEC_ECUDA, cudaGetErrorString(e));
        }
        done_steps += chunk;
        const salec_status st = salec_batch_poll(b, poll.data());
        if (st != SALEC_OK) return st;
        done = 0;
        long tiles_done = 0, tiles_all = 0;
        for (int r = 0; r < n; ++r) {
            const bool d = (poll[5 * r] >= poll[5 * r + 4] || poll[5 * r + 3] != 0.0);
            done += d;
            if (!b->retired[r]) {
                const long t = tiles_of(b->runs[r]->g.nr, b->runs[r]->g.nz, 3, b->shape[3]);
                tiles_all += t;
                if (d) tiles_done += t;
            }
        }
        if (done == n) break;
        // once finished runs hold an eighth of the blocks, leave them out of the work lists
        // (their blocks only return early) and capture the graph again
        if (8 * tiles_done >= tiles_all && tiles_done > 0) {
            for (int r = 0; r < n; ++r)
                if ((poll[5 * r] >= poll[5 * r + 4] || poll[5 * r + 3] != 0.0)) b->retired[r] = 1;
            const salec_status st2 = batch_build_work(b);
            if (st2 != SALEC_OK) return st2;
        }
    }
    if (steps_done) *steps_done = done_steps;
    if (runs_done) *runs_done = done;
    return SALEC_OK;
}

// Persistent mode: one block shape for every phase, chosen by the time of trial_steps
// steps in one launch.
static salec_status batch_autotune_persistent(salec_batch* b, int trial_steps, int* shapes_out)
{
    double best = 1e300;
    dim3 pick = b->shape[0];
    for (int c = 0; c < kNumShapes; ++c) {
        if (kShapes[c].x * kShapes[c].y > (unsigned)kPersistMaxThreads) continue;
        for (int k = 0; k < 6; ++k) b->shape[k] = kShapes[c];
        salec_status st = batch_prepare_persistent(b);
        if (st == SALEC_OK) st = batch_build_work(b);
        b->timing = false;
        if (st == SALEC_OK) st = salec_batch_step(b, 1);
        b->timing = true;
        b->ev_used = 0;
        if (st == SALEC_OK) st = salec_batch_step(b, trial_steps);
        b->timing = false;
        if (st != SALEC_OK) return st;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, SALEC_ECUDA, "sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
        b->ev_used = 0;
        if (ms < best) { best = ms; pick = kShapes[c]; }
    }
    for (int k = 0; k < 6; ++k) b->shape[k] = pick;
    salec_status st = batch_prepare_persistent(b);
    if (st == SALEC_OK) st = batch_build_work(b);
    if (shapes_out)
        for (int k = 0; k < 6; ++k) { shapes_out[2 * k] = (int)pick.x; shapes_out[2 * k + 1] = (int)pick.y; }
    return st;
}

salec_status salec_batch_expire_next_barrier(salec_batch* b)
{
    if (!b || !b->persistent) return SALEC_EINVAL;
    b->expire_next = true;
    return SALEC_OK;
}

salec_status salec_batch_set_persistent(salec_batch* b, int on)
{
    if (!b) return SALEC_EINVAL;
    b->persistent = on != 0;
    if (b->persistent) {
        // every phase takes the block shape of the first kernel (at most kPersistMaxThreads)
        dim3 blk = b->shape[0];
        if (blk.x * blk.y > (unsigned)kPersistMaxThreads) blk = dim3(32, 4);
        for (int k = 0; k < 6; ++k) b->shape[k] = blk;
        b->pgraph = true;
        const salec_status st = batch_prepare_persistent(b);
        if (st != SALEC_OK) { b->persistent = false; return st; }
    }
    return batch_build_work(b);
}

salec_status salec_batch_autotune(salec_batch* b, int trial_steps, int* shapes_out)
{
    HostRange range("salec_batch_autotune");
    if (!b || trial_steps < 1) return SALEC_EINVAL;
    if (b->persistent) return batch_autotune_persistent(b, trial_steps, shapes_out);
    const int K = launches_per_step();
    double best[6];
    dim3 pick[6];
    for (int k = 0; k < K; ++k) { best[k] = 1e300; pick[k] = b->shape[k]; }
    for (int c = 0; c < kNumShapes; ++c) {
        for (int k = 0; k < K; ++k) b->shape[k] = kShapes[c];
        salec_status st = batch_build_work(b);
        if (st != SALEC_OK) return st;
        b->timing = false;
        st = salec_batch_step(b, 1);
        if (st != SALEC_OK) return st;
        b->timing = true;
        b->ev_used = 0;
        st = salec_batch_step(b, trial_steps);
        if (st != SALEC_OK) return st;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, SALEC_ECUDA, "sync");
        for (int k = 0; k < K; ++k) {
            double tot = 0.0;
            for (int s = 0; s < trial_steps; ++s) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, b->ev[(size_t)s * (K + 1) + k], b->ev[(size_t)s * (K + 1) + k + 1]);
                tot += ms;
            }
            if (tot < best[k]) { best[k] = tot; pick[k] = kShapes[c]; }
        }
        b->timing = false;
        b->ev_used = 0;
    }
    for (int k = 0; k < K; ++k) b->shape[k] = pick[k];
    const salec_status st = batch_build_work(b);
    if (shapes_out)
        for (int k = 0; k < K; ++k) { shapes_out[2 * k] = (int)pick[k].x; shapes_out[2 * k + 1] = (int)pick[k].y; }
    return st;
}

const char* salec_batch_last_error(const salec_batch* b) { return b ? b->err.c_str() : "null batch"; }

void salec_batch_destroy(salec_batch* b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

int salec_launches_per_step(const salec_ctx* ctx)
{
    // the Courant, rest-tile and tile kernels; beside the tile kernel: the Courant, scan,
    // copy and tile kernels
    if (ctx && ctx->form == SALEC_STEP_FUSED) return beside(ctx) ? 4 : 3;
    return kernels_per_step();
}

salec_status salec_fused_queue(salec_ctx* ctx, int* queued, int* tiles)
{
    if (!ctx || !queued || !tiles) return SALEC_EINVAL;
    if (!ctx->finalized) return fail(ctx, SALEC_EORDER, "fused_queue before finalize");
    *queued = *tiles = 0;
    if (!ctx->rates_valid) return SALEC_OK;
    // the step that wrote the current copy used the other copy's queue
    TileWork w;
    cudaError_t e = cudaMemcpyAsync(&w, ctx->base + ctx->L.work + (1 - ctx->parity) * sizeof(TileWork), sizeof(w),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "fused queue");
    if (w.next == 0) return SALEC_OK;      // no fused step since the queues were emptied
    *queued = w.count + w.back;
    *tiles = mixed(ctx) ? fused_tiles<float>(ctx->Pf) : fused_tiles<double>(ctx->Pd);
    return SALEC_OK;
}

const char* salec_last_error(const salec_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : noalloc_last_error();
}

void salec_destroy(salec_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (int k = 0; k < 2; ++k)
        if (ctx->fgraph[k]) cudaGraphExecDestroy(ctx->fgraph[k]);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    release_beside(ctx);
    delete ctx;
}

}  // extern "C"
