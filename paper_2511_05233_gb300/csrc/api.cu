// C-ABI layer of libdgls: context setup, parameters of the paper, Newton-GMRES implicit Euler
// steps, time-step controllers and the discharge loop.  Kernels live in dg0.cu, dg1.cu, la.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dgls.h"
#include "internal.h"

using namespace dgls;

// dres[DRES_ONE] holds the constant 1.0 (written once at setup from pageable memory) for
// updates that need a device-side unit coefficient.
constexpr int DRES_ONE = 99;
static const double kOne = 1.0;

struct dg_ctx {
    DevArena arena;                // workspace from a caller buffer (dg_setup_in) or counted (estimate)
    dg_params prm;
    DevParams P;
    Geo G;
    LaunchCtx L;
    int64_t launches = 0;
    int64_t ndof = 0;
    int64_t nblk = 0;              // preconditioner blocks
    int64_t ws_bytes = 0;
    int n_cc = 0;
    std::string err;
    std::vector<void*> allocs;
    // geometry
    uint8_t* d_phase = nullptr;
    int32_t* d_cmap = nullptr;
    int32_t* d_sidx = nullptr;
    // model scratch (transport factors or DG1 face data)
    double* gb = nullptr;
    double* gbd = nullptr;
    float* gb32 = nullptr;
    float* gbd32 = nullptr;
    // preconditioner
    double* blk = nullptr;
    float* blk32 = nullptr;
    int* d_bad = nullptr;
    // Newton vectors
    double *zc = nullptr, *zt = nullptr, *R = nullptr, *Rt = nullptr, *dz = nullptr, *zn = nullptr;
    // Krylov (FP64 or FP32 by precision)
    void* V = nullptr;
    void* w = nullptr;
    void* u = nullptr;
    void* x = nullptr;             // Krylov combination sum y_k V_k
    DG1Lin lin{};                  // linearised FP64 DG1 JVP (cached derivative data)
    bool has_lin = false;
    bool lin_valid = false;        // lin holds the linearisation at the current Newton iterate
    void* y1 = nullptr;            // CPR: potential correction
    void* t2 = nullptr;            // CPR: remaining residual
    std::vector<MGLevel> mg;
    std::vector<MGLevel> mgsp[3];  // species coarse level: one hierarchy per pair of liquid species
    int sp_pairs = 0;
    bool sp_on = false;            // species correction built for the current preconditioner
    float* z32 = nullptr;
    // products of dg_jvp_fused and of the FP32 Krylov loop run the batched kernels with a one-job
    // table (the same compiled kernels as in a batch): a ring of job records, pinned staging and the
    // events that say when the device has read a staging slot
    static constexpr int RING = 4;
    unsigned char* d_ring = nullptr;   // RING x JOB_SLOT bytes
    unsigned char* h_ring = nullptr;
    cudaEvent_t ring_ev[RING] = {};
    int ring_next = 0;
    int2* d_map_self = nullptr;        // (0, b) for every block of this grid (the largest block count of any kind)
    int nblk_fused = 0, nblk_dg0 = 0;
    // discharge work states
    double *za = nullptr, *zb = nullptr, *zC = nullptr, *zF = nullptr;
    // reductions
    double* partial = nullptr;
    double* dres = nullptr;
    double* hres = nullptr;        // pinned host mirror
    double* d_vals = nullptr;      // equilibrium field values
    // statistics of the last step
    int gmres_its = 0, res_evals = 0, jvp_evals = 0;
    int64_t reorth_passes = 0;  // second Gram-Schmidt passes taken (diagnostic)
    // optional per-category kernel timing (CUDA events on the context stream)
    bool prof = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[5] = {0, 0, 0, 0, 0};
    int64_t prof_calls[5] = {0, 0, 0, 0, 0};
};

namespace {
struct ProfScope {
    dg_ctx* c;
    int cat;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(dg_ctx* ctx, int category) : c(ctx), cat(category) {
        if (!c->prof) return;
        a = take();
        b = take();
        if (a && b) cudaEventRecord(a, c->L.st);
    }
    cudaEvent_t take() {
        if (!c->ev_pool.empty()) { cudaEvent_t e = c->ev_pool.back(); c->ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    ~ProfScope() {
        if (!c->prof || !a || !b) return;
        cudaEventRecord(b, c->L.st);
        c->ev.push_back({cat, {a, b}});
    }
};

// Resolve recorded event pairs (the stream must have been synchronised).
void prof_flush(dg_ctx* c) {
    for (auto& e : c->ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess) {
            c->prof_ms[e.first] += ms;
            c->prof_calls[e.first] += 1;
        }
        c->ev_pool.push_back(e.second.first);
        c->ev_pool.push_back(e.second.second);
    }
    c->ev.clear();
}
}  // namespace

static dg_status fail(dg_ctx* c, dg_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e__ = (call);                                                       \
        if (e__ != cudaSuccess)                                                         \
            return fail(ctx, DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

// ------------------------------------------------------------------ paper constants
namespace {
const double F_ = 96485.332, R_ = 8.3145, CREF = 1000.0;
// Tab. 5.1
const double KSP1 = 0.006, KC1 = 120.0, KSP2 = 8e-15, KC2 = 3e-3;
const double U01 = 2.41, U02 = 2.32, U03 = 2.31, U04 = 1.985;
const double KE[6] = {2.53e-6, 3.54e-8, 1.49e-10, 2.05e-7, 9.11e-10, 1.37e-15};
const double AV0 = 94.908e6, RHO_S8 = 2070.4, M_S8 = 0.2565, EPS_S8_0 = 0.095;
const double RHO_LI2S = 1659.0, M_LI2S = 0.0459, EPS_LI2S_0 = 2.77e-6;
const double AV_A = 0.1392, AV_B = 3.310, KAPPA_S = 1.0, K_ANO = 5.0e-3;
// Tab. 5.2 (order: Li+, S8(L), S8^2-, S6^2-, S4^2-, S^2-) and the anion
const double D0_TO[6] = {9.3e-10, 10.0e-10, 5.3e-10, 5.3e-10, 7.6e-10, 0.6e-10};
const double Z_TO[6] = {1, 0, -2, -2, -2, -2};
const double WS_TO[6] = {0, 8, 8, 6, 4, 1};
const double D0_A = 9.3e-10, C_LI_0 = 1500.0;
// Tab. 2 and Sec. 2.1
const double X_CATHODE = 0.168, X_SULFUR = 0.0956, EPS_SEP = 0.4;
const double VISC = 7.76e-4;

// Tab. 6 equilibrium: concentrations (Li+, S8(L), S8^2-, S6^2-, S4^2-, S^2-), Delta Phi_0, U5, U6.
void tab6(double T, double out_c[6], double* dphi0, double* U5, double* U6) {
    const double rtf = R_ * T / F_;
    const double cS8 = KSP1 * CREF;
    const double cS2 = KSP2 * CREF * CREF * CREF / (C_LI_0 * C_LI_0);
    const double d0 = (0.75 * U01 + 0.25 * U02) / 6.0 + U03 / 12.0 + 0.75 * U04 +
                      rtf * (std::log(cS8 / CREF) / 16.0 - 0.5 * std::log(cS2 / CREF));
    const double cS8_2 = cS8 * std::exp(-2.0 * (d0 - U01) / rtf);
    const double cS6_2 = CREF * std::pow(cS8 / CREF, 0.75) * std::exp(-2.0 * (d0 - (0.75 * U01 + 0.25 * U02)) / rtf);
    const double cS4_2 = CREF * std::pow(cS2 / CREF, 4.0) * std::exp(6.0 * (d0 - U04) / rtf);
    *U5 = d0 - rtf * (0.5 * std::log(cS8_2 / CREF) - std::log(cS4_2 / CREF));
    *U6 = d0 - rtf * (std::log(cS4_2 / CREF) / 6.0 + 4.0 / 3.0 * std::log(C_LI_0 / CREF));
    *dphi0 = d0;
    out_c[0] = C_LI_0; out_c[1] = cS8; out_c[2] = cS8_2; out_c[3] = cS6_2; out_c[4] = cS4_2; out_c[5] = cS2;
}
}  // namespace

extern "C" dg_status dg_params_default(dg_params* p, int32_t chemistry, int32_t order) {
    if (!p || (chemistry != 0 && chemistry != 1) || (order != 0 && order != 1)) return DG_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->order = order;
    p->chemistry = chemistry;
    p->T = 298.15;
    p->f_C = 0.5;
    p->j_el = 0.0;
    p->eps_struct = 0.4;
    p->penalty = 1.0;
    p->smooth = 1;
    p->precision = DG_PREC_FP64;
    p->gmres_restart = 30;
    p->gmres_max_it = 600;
    p->newton_rtol = 1e-10;
    p->newton_atol = 1e-12;
    p->preconditioner = 2;
    p->mg_cycles = 1;
    p->precond_every = 0;
    p->reorth = 2;
    p->species_mg = 2;
    p->newton_stall_rtol = 1e-8;
    p->newton_max_it = 25;
    p->eta_max = 1e-2;
    p->eta_min = 1e-3;
    p->hbm_budget_bytes = 0;
    p->jvp_form = 0;
    return DG_OK;
}

// ------------------------------------------------------------------ setup
template <class T>
static cudaError_t dalloc(dg_ctx* ctx, T** ptr, int64_t n) {
    if (n <= 0) n = 1;
    void* q = nullptr;
    cudaError_t e = ctx->arena.active ? arena_alloc(&ctx->arena, (size_t)n * sizeof(T), &q)
                                      : cudaMalloc(&q, (size_t)n * sizeof(T));
    if (e != cudaSuccess) return e;
    if (!ctx->arena.active) ctx->allocs.push_back(q);
    ctx->ws_bytes += n * (int64_t)sizeof(T);
    *ptr = (T*)q;
    return cudaSuccess;
}

static void free_all(dg_ctx* ctx) {
    for (int k = 0; k < dg_ctx::RING; ++k)
        if (ctx->ring_ev[k]) { cudaEventDestroy(ctx->ring_ev[k]); ctx->ring_ev[k] = nullptr; }
    if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
    ctx->h_ring = nullptr;
    for (auto& e : ctx->ev) { ctx->ev_pool.push_back(e.second.first); ctx->ev_pool.push_back(e.second.second); }
    ctx->ev.clear();
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->ev_pool.clear();
    for (void* q : ctx->allocs) cudaFree(q);
    ctx->allocs.clear();
    if (ctx->hres) cudaFreeHost(ctx->hres);
    ctx->hres = nullptr;
}

// Set up a context; with arena the workspaces come from the caller's buffer, and with count the
// allocations are only counted (*count receives the bytes) and no context is returned.
static dg_status setup_impl(const dg_structure* s, const dg_params* prm, void* stream, const DevArena* arena,
                            int64_t* count, dg_ctx** out) {
    if (!out) return DG_ERR_ARG;
    *out = nullptr;
    if (!s || !prm || !s->phase || s->nx < 2 || s->ny < 1 || s->nz < 1 || !(s->h > 0)) return DG_ERR_ARG;
    if ((prm->order != 0 && prm->order != 1) || (prm->chemistry != 0 && prm->chemistry != 1)) return DG_ERR_ARG;
    if (!(prm->eps_struct > 0 && prm->eps_struct <= 1) || prm->gmres_restart < 1 || prm->gmres_restart > MAXK - 1)
        return DG_ERR_ARG;
    if (prm->reorth < 0 || prm->reorth > 2) return DG_ERR_ARG;
    if (prm->species_mg < 0 || prm->species_mg > 2) return DG_ERR_ARG;
    if (prm->preconditioner != 0 && (prm->mg_cycles < 1 || prm->mg_cycles > 16)) return DG_ERR_ARG;
    if (!(prm->newton_stall_rtol >= 0.0)) return DG_ERR_ARG;
    if (prm->jvp_form < 0 || prm->jvp_form > 2) return DG_ERR_ARG;
    const int64_t ncell64 = (int64_t)s->nx * s->ny * s->nz;
    if (ncell64 > 2000000000LL) return DG_ERR_ARG;
    dg_ctx* ctx = new dg_ctx();
    if (arena) ctx->arena = *arena;
    if (count) ctx->arena = DevArena{nullptr, 0, 0, true};
    ctx->prm = *prm;
    ctx->L.st = (cudaStream_t)stream;
    ctx->L.counter = &ctx->launches;
    const int nx = s->nx, ny = s->ny, nz = s->nz, ncell = (int)ncell64;
    // ---- host geometry: phases, compacted structure list
    std::vector<int32_t> cmap(ncell, -1), sidx;
    sidx.reserve(ncell / 2);
    for (int c = 0; c < ncell; ++c) {
        uint8_t ph = s->phase[c];
        if (ph > 2) { delete ctx; return DG_ERR_ARG; }
        if (ph == 1) { cmap[c] = (int32_t)sidx.size(); sidx.push_back(c); }
    }
    int n_cc = 0;
    for (int q = 0; q < ny * nz; ++q)
        if (s->phase[(int64_t)q * nx] == 1) ++n_cc;
    if (n_cc == 0) {
        dg_status st = fail(ctx, DG_ERR_ARG, "no structure voxel touches the current collector");
        delete ctx;
        return st;
    }
    int n_sep = 0;
    for (int i = nx - 1; i >= 0; --i) {
        bool all = true;
        for (int q = 0; q < ny * nz && all; ++q) all = s->phase[(int64_t)q * nx + i] == 2;
        if (!all) break;
        ++n_sep;
    }
    ctx->n_cc = n_cc;
    // ---- device parameters
    DevParams& P = ctx->P;
    std::memset(&P, 0, sizeof(P));
    P.nx = nx; P.ny = ny; P.nz = nz;
    P.n_cell = ncell;
    P.n_struct = (int)sidx.size();
    const bool to = prm->chemistry == DG_CHEM_TRADEOFF;
    P.nl = to ? 6 : 3;
    P.ns = to ? 2 : 0;
    P.nf = P.nl + P.ns + 2;
    P.order = prm->order;
    P.h = s->h;
    P.V = s->h * s->h * s->h;
    P.A = s->h * s->h;
    P.F = F_;
    P.RT = R_ * prm->T;
    P.F_RT = F_ / P.RT;
    P.F_2RT = 0.5 * P.F_RT;
    P.cref = CREF;
    const int spec_to[6] = {0, 1, 2, 3, 4, 5};
    const int spec_r3[3] = {0, 1, 2};
    for (int m = 0; m < P.nl; ++m) {
        int q = to ? spec_to[m] : spec_r3[m];
        P.D0[m] = D0_TO[q];
        P.zc[m] = Z_TO[q];
        P.wS[m] = WS_TO[q];
        P.kappa_m[m] = P.zc[m] * P.F_RT * P.D0[m];
        P.Kd[m] = P.zc[m] * F_ * (P.D0[m] - D0_A);
        P.Km[m] = P.zc[m] * F_ * P.F_RT * (P.zc[m] * P.D0[m] + D0_A);
    }
    P.D0A = D0_A;
    P.visc = VISC;
    const double es = prm->eps_struct;
    P.eps_sep = EPS_SEP;
    P.cbd = (X_CATHODE - X_SULFUR) / es;
    P.eps_frozen[0] = EPS_S8_0 / es;
    P.eps_frozen[1] = EPS_LI2S_0 / es;
    P.aV0p = AV0 / es;
    P.s8ref = 1.2 * EPS_S8_0 / es;
    P.li2sref = AV_A * std::exp(-AV_B * prm->f_C) / es;
    P.rhoM[0] = RHO_S8 / M_S8;
    P.rhoM[1] = RHO_LI2S / M_LI2S;
    P.kappa_s = KAPPA_S;
    P.kAno = K_ANO;
    double j_el = prm->j_el;
    if (!(j_el > 0)) {
        const double c_theo = 16.0 * F_ / M_S8;                       // C/kg (App. B)
        const double L_cat = (nx - n_sep) * s->h;
        j_el = prm->f_C / 3600.0 * c_theo * RHO_S8 * EPS_S8_0 * L_cat;
    }
    P.j_cc = j_el * (double)ny * nz / n_cc;
    P.kC[0] = KC1; P.kC[1] = KC2;
    P.sqK[0] = std::sqrt(KSP1); P.sqK[1] = std::sqrt(KSP2);
    double ceq[6], d0, U5, U6;
    tab6(prm->T, ceq, &d0, &U5, &U6);
    const double U0s[6] = {U01, U02, U03, U04, U5, U6};
    for (int k = 0; k < 6; ++k) {
        P.kE[k] = KE[k];
        P.U0[k] = U0s[k];
        P.eUf[k] = std::exp(P.F_2RT * U0s[k]);
        P.eUb[k] = std::exp(-P.F_2RT * U0s[k]);
    }
    P.penalty = prm->penalty;
    P.smooth = prm->smooth;
    // derived constants (the kernels read them instead of forming them at run time) and their FP32 copies
    P.icref = 1.0 / P.cref;
    P.is8ref = 1.0 / P.s8ref;
    P.ili2sref = 1.0 / P.li2sref;
    for (int q = 0; q < 2; ++q) P.isqK[q] = 1.0 / P.sqK[q];
    for (int k = 0; k < 6; ++k) P.FU2RT[k] = P.F_2RT * P.U0[k];
    P.one_m_cbd = 1.0 - P.cbd;
    P.eps_frozen_sum = P.eps_frozen[0] + P.eps_frozen[1];
    {
        DevParams::F32& f = P.f;
        f.F = (float)P.F; f.F_2RT = (float)P.F_2RT; f.icref = (float)P.icref; f.visc = (float)P.visc;
        f.eps_sep = (float)P.eps_sep; f.one_m_cbd = (float)P.one_m_cbd; f.eps_frozen_sum = (float)P.eps_frozen_sum;
        f.aV0p = (float)P.aV0p; f.is8ref = (float)P.is8ref; f.ili2sref = (float)P.ili2sref;
        for (int m = 0; m < 6; ++m) {
            f.wS[m] = (float)P.wS[m]; f.kE[m] = (float)P.kE[m]; f.FU2RT[m] = (float)P.FU2RT[m];
            f.eUf[m] = (float)P.eUf[m]; f.eUb[m] = (float)P.eUb[m];
        }
        for (int q = 0; q < 2; ++q) {
            f.sqK[q] = (float)P.sqK[q]; f.isqK[q] = (float)P.isqK[q]; f.kC[q] = (float)P.kC[q];
            f.eps_frozen[q] = (float)P.eps_frozen[q];
        }
    }
    const int nn = prm->order == 1 ? 8 : 1;
    const double M = prm->order == 1 ? P.V / 8.0 : P.V;
    int64_t off = 0;
    for (int f = 0; f < P.nf; ++f) {
        bool st = (f >= P.nl && f < P.nl + P.ns) || f == P.nf - 1;
        P.is_struct[f] = st ? 1 : 0;
        P.flen[f] = st ? P.n_struct : P.n_cell;
        P.off[f] = off;
        off += P.flen[f] * nn;
        bool pot = f >= P.nf - 2;
        P.rscale[f] = pot ? 1.0 / (M * F_ * CREF) : 1.0 / (M * CREF);
    }
    ctx->ndof = off;
    // equilibrium field values
    double vals[DG_MAXF];
    if (to) {
        for (int m = 0; m < 6; ++m) vals[m] = ceq[m];
        vals[6] = EPS_S8_0 / es;
        vals[7] = EPS_LI2S_0 / es;
        vals[8] = 0.0;
        vals[9] = d0;
    } else {
        vals[0] = 1000.0; vals[1] = 10.0; vals[2] = 100.0;
        vals[3] = 0.0;
        // Nernst potential of E1 (Eq. 24): U0 - RT/F ln(a_S8^2-^{1/2} / a_S8(L)^{1/2})
        vals[4] = U01 - P.RT / F_ * (0.5 * std::log(vals[2] / CREF) - 0.5 * std::log(vals[1] / CREF));
    }
    // ---- allocations
    const bool mixed = prm->precision == DG_PREC_MIXED;
    const int m = prm->gmres_restart;
    ctx->nblk = (int64_t)ncell * nn;
    const int64_t N = ctx->ndof;
    int64_t scratch = prm->order == 1 ? dg1_face_buffer_len(P) : (int64_t)ncell;
    int64_t need = ncell * (1 + 4 + 4) + N * 8 * (6 + 4) + scratch * 8 * 2 +
                   ctx->nblk * P.nf * P.nf * 8 + (int64_t)(m + 1) * N * (mixed ? 4 : 8) + 3 * N * (mixed ? 4 : 8) +
                   N * 8 + (mixed ? (N * 4 + scratch * 4 * 2 + ctx->nblk * P.nf * P.nf * 4) : 0);
    if (prm->order == 1) {   // the linearisation (FP64, or FP32 for the mixed-precision product)
        int64_t njn, ngam, nface;
        dg1_lin_sizes(P, &njn, &ngam, &nface);
        need += (njn + 2 * ngam + nface + dg1_lin_flux_len(P)) * (mixed ? 4 : 8);
    }
    if (prm->preconditioner != 0) {   // multigrid hierarchies: 153 bytes a voxel on level 0, 8/7 over all levels
        const int hier = 1 + (prm->species_mg != 0 ? (P.nl + 1) / 2 : 0);
        need += hier * ncell * 175;
    }
    if (!count && prm->hbm_budget_bytes > 0 && need > prm->hbm_budget_bytes) {
        dg_status st = fail(ctx, DG_ERR_OOM, "workspace of " + std::to_string(need) + " bytes exceeds hbm_budget_bytes");
        delete ctx;
        return st;
    }
#define AL(ptr, n)                                                        \
    do {                                                                  \
        if (dalloc(ctx, &(ptr), (n)) != cudaSuccess) {                    \
            free_all(ctx);                                                \
            delete ctx;                                                   \
            return DG_ERR_OOM;                                            \
        }                                                                 \
    } while (0)
    AL(ctx->d_phase, ncell);
    AL(ctx->d_cmap, ncell);
    AL(ctx->d_sidx, (int64_t)sidx.size());
    AL(ctx->gb, scratch);
    AL(ctx->gbd, scratch);
    AL(ctx->blk, ctx->nblk * P.nf * P.nf);
    AL(ctx->d_bad, 4);
    AL(ctx->zc, N); AL(ctx->zt, N); AL(ctx->R, N); AL(ctx->Rt, N); AL(ctx->dz, N); AL(ctx->zn, N);
    AL(ctx->za, N); AL(ctx->zb, N); AL(ctx->zC, N); AL(ctx->zF, N);
    AL(ctx->partial, (int64_t)RED_BLOCKS * MAXK + 64);
    ctx->nblk_fused = (ncell + FUSED_VOXELS - 1) / FUSED_VOXELS;
    ctx->nblk_dg0 = (ncell + 127) / 128;
    AL(ctx->d_ring, (int64_t)dg_ctx::RING * JOB_SLOT);
    AL(ctx->d_map_self, std::max(ctx->nblk_fused, ctx->nblk_dg0));
    AL(ctx->dres, 256);
    AL(ctx->d_vals, DG_MAXF);
    if (mixed) {
        float *V, *w, *u, *x, *y1, *t2;
        AL(V, (int64_t)(m + 1) * N); AL(w, N); AL(u, N); AL(x, N); AL(y1, N); AL(t2, N);
        ctx->V = V; ctx->w = w; ctx->u = u; ctx->x = x; ctx->y1 = y1; ctx->t2 = t2;
        AL(ctx->z32, N);
        AL(ctx->gb32, scratch);
        AL(ctx->gbd32, scratch);
        AL(ctx->blk32, ctx->nblk * P.nf * P.nf);   // entry-major ([r * nf + c][block]), see block_invert
    } else {
        double *V, *w, *u, *x, *y1, *t2;
        AL(V, (int64_t)(m + 1) * N); AL(w, N); AL(u, N); AL(x, N); AL(y1, N); AL(t2, N);
        ctx->V = V; ctx->w = w; ctx->u = u; ctx->x = x; ctx->y1 = y1; ctx->t2 = t2;
    }
    if (prm->order == 1) {
        int64_t njn, ngam, nface;
        dg1_lin_sizes(P, &njn, &ngam, &nface);
        if (!mixed) {
            double *jn, *gam, *face, *lgb, *lflux;
            AL(jn, njn); AL(gam, ngam); AL(face, nface); AL(lgb, ngam); AL(lflux, dg1_lin_flux_len(P));
            ctx->lin.jn = jn; ctx->lin.gam = gam; ctx->lin.face = face; ctx->lin.gb = lgb; ctx->lin.gbd = ctx->gbd;
            ctx->lin.flux = lflux;
        } else {
            // FP32 linearisation (from the FP32 copy of z) for the FP32 products and blocks
            float *jn, *gam, *face, *lgb, *lflux;
            AL(jn, njn); AL(gam, ngam); AL(face, nface); AL(lgb, ngam); AL(lflux, dg1_lin_flux_len(P));
            ctx->lin.f32 = true;
            ctx->lin.jn32 = jn; ctx->lin.gam32 = gam; ctx->lin.face32 = face; ctx->lin.gb32 = lgb;
            ctx->lin.gbd32 = ctx->gbd32; ctx->lin.flux32 = lflux;
            ctx->lin.z32 = ctx->z32;
            ctx->lin.ndof = N;
        }
        ctx->has_lin = true;
    }
    if (prm->preconditioner != 0 &&
        mg_levels_alloc(ctx->mg, nx, ny, nz, ctx->allocs, &ctx->ws_bytes, &ctx->arena) != cudaSuccess) {
        free_all(ctx);
        delete ctx;
        return DG_ERR_OOM;
    }
    if (prm->preconditioner != 0 && prm->species_mg != 0) {
        ctx->sp_pairs = (P.nl + 1) / 2;
        for (int k = 0; k < ctx->sp_pairs; ++k)
            if (mg_levels_alloc(ctx->mgsp[k], nx, ny, nz, ctx->allocs, &ctx->ws_bytes, &ctx->arena) != cudaSuccess) {
                free_all(ctx);
                delete ctx;
                return DG_ERR_OOM;
            }
    }
#undef AL
    if (count) {   // sizing only: nothing was allocated
        *count = ctx->arena.used;
        delete ctx;
        return DG_OK;
    }
    if (cudaMallocHost(&ctx->hres, 256 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ring, dg_ctx::RING * JOB_SLOT) != cudaSuccess) {
        free_all(ctx);
        delete ctx;
        return DG_ERR_OOM;
    }
    for (int k = 0; k < dg_ctx::RING; ++k)
        if (cudaEventCreateWithFlags(&ctx->ring_ev[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ctx->ring_ev[k], (cudaStream_t)stream) != cudaSuccess) {
            free_all(ctx);
            delete ctx;
            return DG_ERR_CUDA;
        }
    {
        std::vector<int2> self(std::max(ctx->nblk_fused, ctx->nblk_dg0));
        for (size_t b = 0; b < self.size(); ++b) self[b] = make_int2(0, (int)b);
        if (cudaMemcpy(ctx->d_map_self, self.data(), self.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
            free_all(ctx);
            delete ctx;
            return DG_ERR_CUDA;
        }
    }
    cudaStream_t st = ctx->L.st;
    if (cudaMemcpyAsync(ctx->d_phase, s->phase, ncell, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->d_cmap, cmap.data(), ncell * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (!sidx.empty() && cudaMemcpyAsync(ctx->d_sidx, sidx.data(), sidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemcpyAsync(ctx->d_vals, vals, sizeof(vals), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->dres + DRES_ONE, &kOne, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        free_all(ctx);
        delete ctx;
        return DG_ERR_CUDA;
    }
    ctx->G.phase = ctx->d_phase;
    ctx->G.cmap = ctx->d_cmap;
    ctx->G.sidx = ctx->d_sidx;
    *out = ctx;
    return DG_OK;
}

extern "C" dg_status dg_setup(const dg_structure* s, const dg_params* prm, void* stream, dg_ctx** out) {
    return setup_impl(s, prm, stream, nullptr, nullptr, out);
}

extern "C" dg_status dg_setup_in(const dg_structure* s, const dg_params* prm, void* stream, void* workspace_dev,
                                 int64_t workspace_bytes, dg_ctx** out) {
    if (!workspace_dev || workspace_bytes <= 0 || ((uintptr_t)workspace_dev % 256) != 0) {
        if (out) *out = nullptr;
        return DG_ERR_ARG;
    }
    DevArena a{(char*)workspace_dev, workspace_bytes, 0, true};
    return setup_impl(s, prm, stream, &a, nullptr, out);
}

extern "C" dg_status dg_workspace_estimate(const dg_structure* s, const dg_params* prm, int64_t* bytes) {
    if (!bytes) return DG_ERR_ARG;
    dg_ctx* none = nullptr;
    return setup_impl(s, prm, nullptr, nullptr, bytes, &none);
}

extern "C" dg_status dg_destroy(dg_ctx* ctx) {
    if (!ctx) return DG_ERR_ARG;
    if (ctx->L.st) cudaStreamSynchronize(ctx->L.st);
    else cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
    return DG_OK;
}

extern "C" const char* dg_last_error(const dg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
extern "C" int64_t dg_launch_count(const dg_ctx* ctx) { return ctx ? ctx->launches : 0; }
extern "C" int64_t dg_workspace_bytes(const dg_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }
extern "C" int64_t dg_reorth_count(const dg_ctx* ctx) { return ctx ? ctx->reorth_passes : 0; }

extern "C" dg_status dg_layout(const dg_ctx* ctx, int64_t* n_dof, int32_t* n_fields, int64_t off[10], int64_t len[10]) {
    if (!ctx) return DG_ERR_ARG;
    const int nn = ctx->P.order == 1 ? 8 : 1;
    if (n_dof) *n_dof = ctx->ndof;
    if (n_fields) *n_fields = ctx->P.nf;
    for (int f = 0; f < ctx->P.nf; ++f) {
        if (off) off[f] = ctx->P.off[f];
        if (len) len[f] = ctx->P.flen[f] * nn;
    }
    return DG_OK;
}

// ------------------------------------------------------------------ model calls
static dg_status residual_(dg_ctx* ctx, const double* z, const double* zn, double t, double dt, int relax, double* r) {
    ProfScope ps(ctx, 0);
    cudaError_t e = ctx->P.order == 0 ? dg0_residual(ctx->L, ctx->P, ctx->G, z, zn, t, dt, relax, r, ctx->gb)
                                      : dg1_residual(ctx->L, ctx->P, ctx->G, z, zn, t, dt, relax, r, ctx->gb, ctx->gbd);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("residual: ") + cudaGetErrorString(e));
    ctx->res_evals++;
    return DG_OK;
}

// J v through the kernels for this context: the cached linearisation when it is valid and stored in
// the product's precision (DG1), otherwise forward-mode dual numbers.
// One instance's product through the batched kernels (a one-job table): the record goes to the
// next ring slot once the device has read that slot's previous upload.
template <class S>
static cudaError_t fused_self(dg_ctx* ctx, const S* z, const S* v, double t, double dt, int relax, double sc_dt, S* out,
                              S* gb, S* gbd) {
    const bool f32 = std::is_same<S, float>::value;
    const int k = ctx->ring_next;
    ctx->ring_next = (k + 1) % dg_ctx::RING;
    cudaError_t e = cudaEventSynchronize(ctx->ring_ev[k]);
    if (e != cudaSuccess) return e;
    unsigned char* h = ctx->h_ring + (size_t)k * JOB_SLOT;
    unsigned char* d = ctx->d_ring + (size_t)k * JOB_SLOT;
    size_t bytes;
    if (ctx->P.order == 1) {
        dg1_fused_job(f32, ctx->P, ctx->G, z, v, t, dt, relax, sc_dt, out, h);
        bytes = dg1_job_bytes(f32);
    } else {
        Job0<S>* J = reinterpret_cast<Job0<S>*>(h);
        std::memset((void*)J, 0, sizeof(*J));
        J->p = ctx->P;
        J->g = ctx->G;
        J->z = z;
        J->v = v;
        J->gb = gb;
        J->gbd = gbd;
        J->out = out;
        J->t = t;
        J->dt = dt;
        J->sc_dt = sc_dt;
        J->relax = relax;
        bytes = sizeof(Job0<S>);
    }
    if ((e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, ctx->L.st)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ctx->ring_ev[k], ctx->L.st)) != cudaSuccess) return e;
    const bool to = ctx->P.nf == 10;
    if (ctx->P.order == 1) return dg1_jvp_fused_batched(ctx->L, f32, to, d, ctx->d_map_self, ctx->nblk_fused);
    return dg0_batch<S>(ctx->L, to, 1, (const Job0<S>*)d, ctx->d_map_self, ctx->nblk_dg0, 128);
}

template <class S>
static bool use_fused(const dg_ctx* ctx) {
    return ctx->P.order == 1 && (ctx->prm.jvp_form == 2 || (ctx->prm.jvp_form == 0 && std::is_same<S, float>::value));
}

template <class S>
static cudaError_t jvp_kernels(dg_ctx* ctx, const S* z, const S* v, double t, double dt, int relax, double sc_dt, S* out,
                               S* gb, S* gbd) {
    if (use_fused<S>(ctx)) return fused_self<S>(ctx, z, v, t, dt, relax, sc_dt, out, gb, gbd);
    if (ctx->has_lin && ctx->lin_valid && std::is_same<S, float>::value == ctx->lin.f32)
        return dg1_lin_apply<S>(ctx->L, ctx->P, ctx->G, z, v, t, dt, relax, sc_dt, out, ctx->lin);
    return ctx->P.order == 0 ? dg0_jvp<S>(ctx->L, ctx->P, ctx->G, z, v, t, dt, relax, sc_dt, out, gb, gbd)
                             : dg1_jvp<S>(ctx->L, ctx->P, ctx->G, z, v, t, dt, relax, sc_dt, out, gb, gbd);
}

template <class S>
static dg_status jvp_(dg_ctx* ctx, const S* z, const S* v, double t, double dt, int relax, double sc_dt, S* out,
                      S* gb, S* gbd) {
    ProfScope ps(ctx, 1);
    cudaError_t e = jvp_kernels<S>(ctx, z, v, t, dt, relax, sc_dt, out, gb, gbd);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("jvp: ") + cudaGetErrorString(e));
    ctx->jvp_evals++;
    return DG_OK;
}

// Diagonal blocks of S J (in FP32 arithmetic when the Krylov loop is FP32: they only precondition),
// their inverses, and the potential multigrid hierarchy at z.
static dg_status build_precond(dg_ctx* ctx, const double* z, double t, double dt, int relax) {
    ProfScope ps(ctx, 2);
    cudaError_t e;
    if (ctx->has_lin && !ctx->lin_valid) return fail(ctx, DG_ERR_ARG, "blocks: no linearisation at this state");
    if (ctx->prm.precision == DG_PREC_MIXED) {
        e = to_f32(ctx->L, ctx->z32, z, ctx->ndof);
        if (e == cudaSuccess) {
            if (ctx->has_lin)   // DG1: blocks from the FP32 linearisation, inverted to FP32 below
                e = dg1_lin_blocks(ctx->L, ctx->P, ctx->G, z, dt, relax, ctx->lin, ctx->blk);
            else
                e = dg0_blocks<float>(ctx->L, ctx->P, ctx->G, ctx->z32, t, dt, relax, ctx->blk, ctx->gb32);
        }
        if (e == cudaSuccess && ctx->prm.preconditioner != 0)   // FP64 transport factors for the multigrid
            e = ctx->P.order == 0 ? dg0_gfactor(ctx->L, ctx->P, ctx->G, z, ctx->gb)
                                  : dg1_gfactor(ctx->L, ctx->P, ctx->G, z, ctx->gb);
    } else if (ctx->has_lin) {
        // FP64 DG1: the blocks come from the linearisation at z, which the caller has just built
        e = dg1_lin_blocks(ctx->L, ctx->P, ctx->G, z, dt, relax, ctx->lin, ctx->blk);
    } else {   // DG0 (every DG1 context carries a linearisation)
        e = dg0_blocks<double>(ctx->L, ctx->P, ctx->G, z, t, dt, relax, ctx->blk, ctx->gb);
    }
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("blocks: ") + cudaGetErrorString(e));
    e = cudaMemsetAsync(ctx->d_bad, 0, sizeof(int), ctx->L.st);
    if (e == cudaSuccess) e = block_invert(ctx->L, ctx->blk, ctx->nblk, ctx->P.nf, ctx->blk32, ctx->d_bad);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("block inverse: ") + cudaGetErrorString(e));
    if (ctx->prm.preconditioner != 0) {
        const double* gbz = (ctx->has_lin && !ctx->lin.f32) ? ctx->lin.gb : ctx->gb;
        e = mg_setup(ctx->L, ctx->P, ctx->G, z, gbz, t, dt, relax, ctx->mg);
        if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("multigrid setup: ") + cudaGetErrorString(e));
    }
    // species coarse level: off while relaxing (the species rows are storage alone there)
    ctx->sp_on = false;
    if (ctx->sp_pairs > 0 && !relax) {
        double dmax = 0.0;
        for (int m = 0; m < ctx->P.nl; ++m) dmax = std::max(dmax, ctx->P.D0[m]);
        ctx->sp_on = ctx->prm.species_mg == 1 || dmax * dt / (ctx->P.h * ctx->P.h) >= 10.0;
    }
    if (ctx->sp_on) {
        const double* gbz = (ctx->has_lin && !ctx->lin.f32) ? ctx->lin.gb : ctx->gb;
        const void* jn = !ctx->has_lin ? nullptr : ctx->lin.f32 ? (const void*)ctx->lin.jn32 : (const void*)ctx->lin.jn;
        e = mg_species_setup(ctx->L, ctx->P, ctx->G, z, gbz, jn, ctx->lin.f32, t, dt, ctx->mgsp, ctx->sp_pairs);
        if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("species multigrid setup: ") + cudaGetErrorString(e));
    }
    return DG_OK;
}

// u = M^{-1} v: block Jacobi, or the two-stage CPR preconditioner
//   y1 = P MG(R v) (+ the species coarse correction);  u = B^{-1} (v - S J y1) + y1
template <class S>
static dg_status precond_apply_(dg_ctx* ctx, const S* v, S* u, const S* zS, double t, double dt, int relax, S* gbS,
                                S* gbdS, const void* blkS) {
    ProfScope ps(ctx, 3);
    const int64_t N = ctx->ndof;
    if (ctx->prm.preconditioner == 0) {
        CK(block_apply<S>(ctx->L, ctx->P, ctx->G, blkS, v, u));
        return DG_OK;
    }
    S* y1 = (S*)ctx->y1;
    S* t2 = (S*)ctx->t2;
    CK(cpr_stage1<S>(ctx->L, ctx->P, ctx->G, ctx->mg, ctx->prm.mg_cycles, v, y1));
    // with the species coarse level the two corrections are always applied in the multiplicative
    // form: added to the node blocks, the decoupled species correction over-corrects the smooth
    // modes of the reaction-coupled polysulfides wherever storage and diffusion are comparable
    if (ctx->sp_on) CK(mg_species_apply<S>(ctx->L, ctx->P, ctx->mgsp, ctx->sp_pairs, v, y1));
    if (ctx->prm.preconditioner == 2 && !ctx->sp_on) {
        // additive form: u = B^{-1} v + P MG(R v) (no Jacobian-vector product)
        CK(block_apply<S>(ctx->L, ctx->P, ctx->G, blkS, v, u));
        CK(saxpby<S>(ctx->L, u, 1.0, y1, 1.0, N));
        return DG_OK;
    }
    cudaError_t e = jvp_kernels<S>(ctx, zS, y1, t, dt, relax, dt, t2, gbS, gbdS);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("jvp: ") + cudaGetErrorString(e));
    ctx->jvp_evals++;
    CK(saxpby<S>(ctx->L, t2, -1.0, v, 1.0, N));
    CK(block_apply<S>(ctx->L, ctx->P, ctx->G, blkS, t2, u));
    CK(saxpby<S>(ctx->L, u, 1.0, y1, 1.0, N));
    return DG_OK;
}

static dg_status sync_(dg_ctx* ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->L.st);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
    if (ctx->prof) prof_flush(ctx);
    return DG_OK;
}

extern "C" dg_status dg_profile(dg_ctx* ctx, int32_t enable) {
    if (!ctx) return DG_ERR_ARG;
    dg_status s = sync_(ctx);
    if (s != DG_OK) return s;
    ctx->prof = enable != 0;
    for (int k = 0; k < 5; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_calls[k] = 0; }
    return DG_OK;
}

extern "C" dg_status dg_profile_read(const dg_ctx* ctx, double ms[5], int64_t calls[5]) {
    if (!ctx || !ms || !calls) return DG_ERR_ARG;
    for (int k = 0; k < 5; ++k) { ms[k] = ctx->prof_ms[k]; calls[k] = ctx->prof_calls[k]; }
    return DG_OK;
}

static dg_status scaled_norm_(dg_ctx* ctx, const double* r, double dt, double* out) {
    cudaError_t e = scaled_norm2(ctx->L, ctx->P, r, dt, ctx->partial, ctx->dres + 200);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->hres + 200, ctx->dres + 200, sizeof(double), cudaMemcpyDeviceToHost, ctx->L.st);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("norm: ") + cudaGetErrorString(e));
    dg_status s = sync_(ctx);
    if (s != DG_OK) return s;
    *out = std::sqrt(ctx->hres[200]);
    return DG_OK;
}

extern "C" dg_status dg_residual(dg_ctx* ctx, const double* z, const double* zold, double t, double dt, double* r) {
    if (!ctx || !z || !zold || !r || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_residual: bad argument");
    return residual_(ctx, z, zold, t, dt, 0, r);
}

extern "C" dg_status dg_jvp(dg_ctx* ctx, const double* z, double t, double dt, const double* v, double* jv) {
    if (!ctx || !z || !v || !jv || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_jvp: bad argument");
    if (ctx->has_lin && !ctx->lin.f32) {   // FP64 product from the FP64 linearisation (else dual numbers)
        CK(dg1_linearize(ctx->L, ctx->P, ctx->G, z, t, dt, 0, ctx->lin));
        ctx->lin_valid = true;
    }
    dg_status s = jvp_<double>(ctx, z, v, t, dt, 0, 0.0, jv, ctx->gb, ctx->gbd);
    ctx->lin_valid = false;
    return s;
}

extern "C" dg_status dg_jvp_fused(dg_ctx* ctx, const double* z, double t, double dt, int32_t precision, const void* v,
                                  void* jv) {
    if (!ctx || !z || !v || !jv || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_jvp_fused: bad argument");
    if (precision == DG_PREC_FP64) {
        ProfScope ps(ctx, 1);
        CK(fused_self<double>(ctx, z, (const double*)v, t, dt, 0, 0.0, (double*)jv, ctx->gb, ctx->gbd));
        return DG_OK;
    }
    if (precision != DG_PREC_MIXED) return fail(ctx, DG_ERR_ARG, "dg_jvp_fused: precision must be FP64 or MIXED");
    if (ctx->prm.precision != DG_PREC_MIXED || !ctx->z32)
        return fail(ctx, DG_ERR_ARG, "dg_jvp_fused: an FP32 product needs a context set up with DG_PREC_MIXED");
    CK(to_f32(ctx->L, ctx->z32, z, ctx->ndof));
    ProfScope ps(ctx, 1);
    CK(fused_self<float>(ctx, ctx->z32, (const float*)v, t, dt, 0, 0.0, (float*)jv, ctx->gb32, ctx->gbd32));
    return DG_OK;
}

extern "C" dg_status dg_block_jacobi(dg_ctx* ctx, const double* z, double t, double dt, const double* v, double* out) {
    if (!ctx || !z || !v || !out || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_block_jacobi: bad argument");
    if (ctx->has_lin) {
        CK(dg1_linearize(ctx->L, ctx->P, ctx->G, z, t, dt, 0, ctx->lin));
        ctx->lin_valid = true;
    }
    dg_status s = build_precond(ctx, z, t, dt, 0);
    ctx->lin_valid = false;
    if (s != DG_OK) return s;
    CK(block_apply<double>(ctx->L, ctx->P, ctx->G, ctx->blk, v, out));
    return DG_OK;
}

extern "C" dg_status dg_limit(dg_ctx* ctx, double* z) {
    if (!ctx || !z) return fail(ctx, DG_ERR_ARG, "dg_limit: bad argument");
    if (ctx->P.order != 1) return fail(ctx, DG_ERR_ARG, "dg_limit: the slope limiter acts on DG1 states");
    CK(dg1_limit(ctx->L, ctx->P, ctx->G, z, ctx->gbd));
    return DG_OK;
}

extern "C" dg_status dg_row_scales(dg_ctx* ctx, double dt, double* s) {
    if (!ctx || !s || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_row_scales: bad argument");
    CK(row_scales(ctx->L, ctx->P, dt, s));
    return DG_OK;
}

extern "C" dg_status dg_equilibrium_state(dg_ctx* ctx, double* z) {
    if (!ctx || !z) return fail(ctx, DG_ERR_ARG, "dg_equilibrium_state: bad argument");
    CK(fill_equilibrium(ctx->L, ctx->P, ctx->d_vals, z));
    return DG_OK;
}

extern "C" dg_status dg_cell_voltage(dg_ctx* ctx, const double* z, double* U) {
    if (!ctx || !z || !U) return fail(ctx, DG_ERR_ARG, "dg_cell_voltage: bad argument");
    CK(cell_voltage(ctx->L, ctx->P, ctx->G, z, ctx->partial, ctx->dres + 210));
    CK(cudaMemcpyAsync(ctx->hres + 210, ctx->dres + 210, sizeof(double), cudaMemcpyDeviceToHost, ctx->L.st));
    dg_status s = sync_(ctx);
    if (s != DG_OK) return s;
    *U = ctx->hres[210];
    return DG_OK;
}

extern "C" dg_status dg_ledger(dg_ctx* ctx, const double* z, double out[5]) {
    if (!ctx || !z || !out) return fail(ctx, DG_ERR_ARG, "dg_ledger: bad argument");
    CK(ledger(ctx->L, ctx->P, ctx->G, z, ctx->partial, ctx->dres + 220));
    CK(cudaMemcpyAsync(ctx->hres + 220, ctx->dres + 220, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->L.st));
    dg_status s = sync_(ctx);
    if (s != DG_OK) return s;
    for (int k = 0; k < 5; ++k) out[k] = ctx->hres[220 + k];
    return DG_OK;
}

// ------------------------------------------------------------------ GMRES
// Right-preconditioned restarted GMRES(m) for (S J) d = b with classical Gram-Schmidt and one
// re-orthogonalisation pass; S the Newton row scales, preconditioner the inverted diagonal
// blocks of S J.  b = -S R(z) is formed from ctx->R.  The correction is accumulated in ctx->dz.
template <class S>
static dg_status gmres_(dg_ctx* ctx, const double* z, double t, double dt, int relax, double eta, int* its_out) {
    const int64_t N = ctx->ndof;
    const int m = ctx->prm.gmres_restart;
    const LaunchCtx& L = ctx->L;
    S* V = (S*)ctx->V;
    S* w = (S*)ctx->w;
    S* u = (S*)ctx->u;
    S* x = (S*)ctx->x;
    const bool mixed = std::is_same<S, float>::value;
    const S* zS = mixed ? (const S*)ctx->z32 : (const S*)z;
    S* gbS = mixed ? (S*)ctx->gb32 : (S*)ctx->gb;
    S* gbdS = mixed ? (S*)ctx->gbd32 : (S*)ctx->gbd;
    const void* blkS = mixed ? (const void*)ctx->blk32 : (const void*)ctx->blk;
    if (mixed) CK(to_f32(L, ctx->z32, z, N));
    CK(cudaMemsetAsync(ctx->dz, 0, N * sizeof(double), L.st));
    double beta0 = -1.0;
    int total = 0;
    std::vector<double> H((m + 1) * m), cs(m), sn(m), gvec(m + 1), y(m);
    const int max_it = ctx->prm.gmres_max_it;
    bool converged = false;
    for (int cycle = 0; total < max_it && !converged; ++cycle) {
        // residual of the current correction: r = b - A dz = -S R - S J dz
        if (cycle == 0) {
            CK(neg_scaled<S>(L, ctx->P, ctx->R, dt, w));
        } else {
            if (mixed) CK(to_f32(L, (float*)u, ctx->dz, N));
            else CK(cudaMemcpyAsync(u, ctx->dz, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
            dg_status s = jvp_<S>(ctx, zS, u, t, dt, relax, dt, x, gbS, gbdS);
            if (s != DG_OK) return s;
            CK(neg_scaled<S>(L, ctx->P, ctx->R, dt, w));
            CK(maxpy<S>(L, w, x, N, N, 1, ctx->dres + DRES_ONE, -1.0));
        }
        CK(mdot<S>(L, w, N, N, 1, w, ctx->partial, ctx->dres + 64));
        CK(scale_copy<S>(L, V, w, N, ctx->dres + 64, 1.0));
        CK(cudaMemcpyAsync(ctx->hres + 64, ctx->dres + 64, sizeof(double), cudaMemcpyDeviceToHost, L.st));
        dg_status s = sync_(ctx);
        if (s != DG_OK) return s;
        double beta = std::sqrt(ctx->hres[64]);
        if (!std::isfinite(beta)) return fail(ctx, DG_ERR_NONFINITE, "GMRES: non-finite residual");
        if (beta0 < 0) beta0 = beta;
        if (beta <= eta * beta0 || beta == 0.0) { converged = true; break; }
        std::fill(gvec.begin(), gvec.end(), 0.0);
        gvec[0] = beta;
        int j = 0;
        for (; j < m && total < max_it; ++j) {
            S* vj = V + (int64_t)j * N;
            s = precond_apply_<S>(ctx, vj, u, zS, t, dt, relax, gbS, gbdS, blkS);
            if (s != DG_OK) return s;
            s = jvp_<S>(ctx, zS, u, t, dt, relax, dt, w, gbS, gbdS);
            if (s != DG_OK) return s;
            // classical Gram-Schmidt: h = V^T w (with ||w||^2 in dres[j+1]), w -= V h (with ||w||^2
            // in dres[64]); a second pass when the first cancelled (reorth = 0) or always (reorth = 1)
            {
                ProfScope ps(ctx, 4);
                CK(mdot<S>(L, V, N, N, j + 1, w, ctx->partial, ctx->dres, true));
                CK(maxpy_norm<S>(L, w, V, N, N, j + 1, ctx->dres, ctx->partial, ctx->dres + 64));
            }
            CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 65 * sizeof(double), cudaMemcpyDeviceToHost, L.st));
            s = sync_(ctx);
            if (s != DG_OK) return s;
            for (int i = 0; i <= j; ++i) H[i * m + j] = ctx->hres[i];
            if (ctx->prm.reorth == 1 || (ctx->prm.reorth == 0 && ctx->hres[64] < 0.5 * ctx->hres[j + 1])) {
                {
                    ProfScope ps(ctx, 4);
                    CK(mdot<S>(L, V, N, N, j + 1, w, ctx->partial, ctx->dres + 32));
                    CK(maxpy_norm<S>(L, w, V, N, N, j + 1, ctx->dres + 32, ctx->partial, ctx->dres + 64));
                }
                CK(cudaMemcpyAsync(ctx->hres + 32, ctx->dres + 32, 33 * sizeof(double), cudaMemcpyDeviceToHost, L.st));
                s = sync_(ctx);
                if (s != DG_OK) return s;
                for (int i = 0; i <= j; ++i) H[i * m + j] += ctx->hres[32 + i];
                ++ctx->reorth_passes;
            }
            {
                ProfScope ps(ctx, 4);
                CK(scale_copy<S>(L, V + (int64_t)(j + 1) * N, w, N, ctx->dres + 64, 1.0));
            }
            ++total;
            double hn = std::sqrt(ctx->hres[64]);
            if (!std::isfinite(hn)) return fail(ctx, DG_ERR_NONFINITE, "GMRES: non-finite Krylov vector");
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], b = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * b;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            double a = H[j * m + j], b = H[(j + 1) * m + j];
            double r = std::hypot(a, b);
            cs[j] = r > 0 ? a / r : 1.0;
            sn[j] = r > 0 ? b / r : 0.0;
            H[j * m + j] = r;
            H[(j + 1) * m + j] = 0.0;
            gvec[j + 1] = -sn[j] * gvec[j];
            gvec[j] = cs[j] * gvec[j];
            if (std::fabs(gvec[j + 1]) <= eta * beta0 || hn == 0.0) { ++j; converged = true; break; }
        }
        // y = H^{-1} g (upper triangular j x j), x = sum y_k V_k, dz += M^{-1} x
        for (int i = j - 1; i >= 0; --i) {
            double acc = gvec[i];
            for (int k = i + 1; k < j; ++k) acc -= H[i * m + k] * y[k];
            y[i] = H[i * m + i] != 0.0 ? acc / H[i * m + i] : 0.0;
        }
        // hres[100..] is written only here, after the sync that ended the previous cycle, so the
        // asynchronous copy below never reads a slot the host is rewriting
        for (int i = 0; i < j; ++i) ctx->hres[100 + i] = y[i];
        CK(cudaMemcpyAsync(ctx->dres + 100, ctx->hres + 100, j * sizeof(double), cudaMemcpyHostToDevice, L.st));
        CK(cudaMemsetAsync(x, 0, N * sizeof(S), L.st));
        CK(maxpy<S>(L, x, V, N, N, j, ctx->dres + 100, 1.0));
        s = precond_apply_<S>(ctx, x, u, zS, t, dt, relax, gbS, gbdS, blkS);
        if (s != DG_OK) return s;
        if (mixed) CK(to_f64_add(L, ctx->dz, (const float*)u, 1.0, N));
        else CK(axpby(L, ctx->dz, 1.0, (const double*)u, 1.0, N));
        s = sync_(ctx);
        if (s != DG_OK) return s;
    }
    *its_out = total;
    return DG_OK;
}

// ------------------------------------------------------------------ Newton
// Solve R(z; z^n, t1, dt) = 0 starting from z = zstart (ctx->zc holds the iterate).
static dg_status newton_(dg_ctx* ctx, const double* zn, double t1, double dt, int relax, dg_step_info* info) {
    const int64_t N = ctx->ndof;
    const LaunchCtx& L = ctx->L;
    ctx->gmres_its = 0;
    ctx->res_evals = 0;
    ctx->jvp_evals = 0;
    dg_status s = residual_(ctx, ctx->zc, zn, t1, dt, relax, ctx->R);
    if (s != DG_OK) return s;
    double nrm;
    s = scaled_norm_(ctx, ctx->R, dt, &nrm);
    if (s != DG_OK) return s;
    const double n0 = nrm;
    if (info) { info->norm0 = n0; info->norm = n0; info->converged = 0; info->newton_iterations = 0; }
    if (!std::isfinite(nrm)) return fail(ctx, DG_ERR_NONFINITE, "non-finite initial residual");
    double eta = ctx->prm.eta_max;
    const bool mixed = ctx->prm.precision == DG_PREC_MIXED;
    int it = 0;
    dg_status result = DG_OK;
    const double floor_ = ctx->prm.newton_atol * std::sqrt((double)N);
    for (;;) {
        if (nrm <= std::max(ctx->prm.newton_rtol * n0, floor_) || nrm == 0.0) break;
        if (it >= ctx->prm.newton_max_it) { result = fail(ctx, DG_ERR_NOCONV, "Newton: iteration limit"); break; }
        if (ctx->has_lin) {
            ProfScope ps(ctx, 2);
            CK(dg1_linearize(ctx->L, ctx->P, ctx->G, ctx->zc, t1, dt, relax, ctx->lin));
            ctx->lin_valid = true;
        }
        const int every = ctx->prm.precond_every;
        if (it == 0 || (every > 0 && it % every == 0)) {
            s = build_precond(ctx, ctx->zc, t1, dt, relax);
            if (s != DG_OK) return s;
        }
        int its = 0;
        // forcing term never asks for more than the Newton tolerance needs
        double eta_eff = std::max(eta, 0.5 * ctx->prm.newton_rtol * n0 / nrm);
        eta_eff = std::min(eta_eff, ctx->prm.eta_max);
        s = mixed ? gmres_<float>(ctx, ctx->zc, t1, dt, relax, std::max(eta_eff, 1e-6), &its)
                  : gmres_<double>(ctx, ctx->zc, t1, dt, relax, eta_eff, &its);
        ctx->lin_valid = false;
        if (s != DG_OK) return s;
        ctx->gmres_its += its;
        // backtracking line search on ||S R||
        double lam = 1.0, nt = 0.0;
        bool ok = false;
        for (int cut = 0; cut <= 10; ++cut) {
            CK(cudaMemcpyAsync(ctx->zt, ctx->zc, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
            CK(axpby(L, ctx->zt, 1.0, ctx->dz, lam, N));
            s = residual_(ctx, ctx->zt, zn, t1, dt, relax, ctx->Rt);
            if (s != DG_OK) return s;
            s = scaled_norm_(ctx, ctx->Rt, dt, &nt);
            if (s != DG_OK) return s;
            if (std::isfinite(nt) && nt <= (1.0 - 1e-4 * lam) * nrm) { ok = true; break; }
            lam *= 0.5;
        }
        if (!ok) {
            // stagnation at the rounding level of the scaled residual: converged if within the
            // stall tolerance, otherwise a genuine failure
            if (std::isfinite(nrm) && nrm <= ctx->prm.newton_stall_rtol * n0) break;
            result = fail(ctx, DG_ERR_NOCONV, "Newton: line search failed");
            break;
        }
        std::swap(ctx->zc, ctx->zt);
        std::swap(ctx->R, ctx->Rt);
        // stagnation at the rounding level: within the stall tolerance, an iteration that no longer
        // halves ||S R|| has met the floor that rounding puts under the scaled residual (above it
        // the inexact Newton iteration contracts by its forcing term, at most eta_max), so the
        // solve ends here, certified to the same level as a stalled line search
        const bool stagnant = nt <= ctx->prm.newton_stall_rtol * n0 && nt > 0.5 * nrm;
        // Eisenstat-Walker choice 2 (gamma 0.9, alpha 2) with the usual safeguard
        double eta_new = 0.9 * (nt / nrm) * (nt / nrm);
        double safe = 0.9 * eta * eta;
        if (safe > 0.1) eta_new = std::max(eta_new, safe);
        eta = std::min(ctx->prm.eta_max, std::max(ctx->prm.eta_min, eta_new));
        nrm = nt;
        ++it;
        if (stagnant) break;
    }
    if (info) {
        info->converged = result == DG_OK;
        info->newton_iterations = it;
        info->gmres_iterations = ctx->gmres_its;
        info->residual_evals = ctx->res_evals;
        info->jvp_evals = ctx->jvp_evals;
        info->norm = nrm;
    }
    return result;
}

extern "C" dg_status dg_step(dg_ctx* ctx, const double* zn, double* z, double t, double dt, dg_step_info* info) {
    if (!ctx || !zn || !z || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_step: bad argument");
    const int64_t N = ctx->ndof;
    CK(cudaMemcpyAsync(ctx->zn, zn, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
    CK(cudaMemcpyAsync(ctx->zc, zn, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
    dg_status s = newton_(ctx, ctx->zn, t + dt, dt, 0, info);
    if (s != DG_OK && s != DG_ERR_NOCONV) return s;
    CK(cudaMemcpyAsync(z, ctx->zc, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
    dg_status s2 = sync_(ctx);
    return s != DG_OK ? s : s2;
}

extern "C" dg_status dg_step_host(dg_ctx* ctx, const double* zn_host, double* z_host, double t, double dt,
                                  dg_step_info* info) {
    if (!ctx || !zn_host || !z_host || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_step_host: bad argument");
    const int64_t N = ctx->ndof;
    CK(cudaMemcpyAsync(ctx->za, zn_host, N * sizeof(double), cudaMemcpyHostToDevice, ctx->L.st));
    dg_status s = dg_step(ctx, ctx->za, ctx->zb, t, dt, info);
    if (s != DG_OK && s != DG_ERR_NOCONV) return s;
    CK(cudaMemcpyAsync(z_host, ctx->zb, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->L.st));
    dg_status s2 = sync_(ctx);
    return s != DG_OK ? s : s2;
}

extern "C" dg_status dg_relax(dg_ctx* ctx, double* z, double dt, int32_t n_steps) {
    if (!ctx || !z || !(dt > 0) || n_steps < 0) return fail(ctx, DG_ERR_ARG, "dg_relax: bad argument");
    const int64_t N = ctx->ndof;
    double t = 0.0;
    for (int k = 0; k < n_steps; ++k) {
        CK(cudaMemcpyAsync(ctx->zn, z, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
        CK(cudaMemcpyAsync(ctx->zc, z, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
        dg_step_info info;
        dg_status s = newton_(ctx, ctx->zn, t + dt, dt, 1, &info);
        if (s != DG_OK) return s;
        CK(cudaMemcpyAsync(z, ctx->zc, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->L.st));
        t += dt;
    }
    return sync_(ctx);
}

// ------------------------------------------------------------------ discharge
// One implicit Euler attempt from `from` (device) to `to` (device).
static dg_status attempt_(dg_ctx* ctx, const double* from, double* to, double t, double dt, dg_step_info* info) {
    return dg_step(ctx, from, to, t, dt, info);
}

static double rel_err_(dg_ctx* ctx, const double* zF, const double* zC, dg_status* st) {
    // ||zF - zC|| / ||zF|| with the deterministic reductions
    const int64_t N = ctx->ndof;
    const LaunchCtx& L = ctx->L;
    *st = DG_OK;
    if (cudaMemcpyAsync(ctx->zt, zF, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st) != cudaSuccess ||
        axpby(L, ctx->zt, 1.0, zC, -1.0, N) != cudaSuccess ||
        mdot<double>(L, ctx->zt, N, N, 1, ctx->zt, ctx->partial, ctx->dres + 230) != cudaSuccess ||
        mdot<double>(L, zF, N, N, 1, zF, ctx->partial, ctx->dres + 231) != cudaSuccess ||
        cudaMemcpyAsync(ctx->hres + 230, ctx->dres + 230, 2 * sizeof(double), cudaMemcpyDeviceToHost, L.st) != cudaSuccess) {
        *st = fail(ctx, DG_ERR_CUDA, "error estimate failed");
        return 0.0;
    }
    *st = sync_(ctx);
    return std::sqrt(ctx->hres[230] / ctx->hres[231]);
}

extern "C" dg_status dg_discharge(dg_ctx* ctx, double* z, const dg_discharge_opts* o, dg_curve* out) {
    if (!ctx || !z || !o || !out || out->n_max < 1 || !out->t || !out->dt || !out->U_cell || !out->c_m)
        return fail(ctx, DG_ERR_ARG, "dg_discharge: bad argument");
    const int64_t N = ctx->ndof;
    const LaunchCtx& L = ctx->L;
    const double c_theo_ah = 16.0 * F_ / M_S8 / 3600.0;
    out->n = 0;
    out->attempts = 0;
    out->failures = 0;
    out->status = DG_OK;
    double t = o->t0, dt = o->dt0;
    double* cur = ctx->za;
    double* nxt = ctx->zb;
    CK(cudaMemcpyAsync(cur, z, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    int sct = 0, halv = 0, n = 0;
    const int max_h = o->max_halvings > 0 ? o->max_halvings : 30;
    const double t_end = o->t_end > 0 ? o->t_end : INFINITY;
    const int max_steps = std::min(o->max_steps > 0 ? o->max_steps : out->n_max, out->n_max);
    double err_prev = o->tol, dt_prev = dt;
    if (o->resume) {   // continue a checkpointed run
        if (!(o->resume->dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_discharge: resume record with dt <= 0");
        t = o->resume->t;
        dt = o->resume->dt;
        err_prev = o->resume->err_prev;
        dt_prev = o->resume->dt_prev;
        sct = o->resume->sct;
        halv = o->resume->halvings;
    }
    dg_status result = DG_OK;
    while (n < max_steps && t < t_end) {
        dg_step_info info;
        std::memset(&info, 0, sizeof(info));
        bool ok = false;
        double lim = 1.0;
        if (o->replay_dt) {
            if (n >= o->n_replay) break;
            dt = o->replay_dt[n];
        }
        if (o->controller == DG_CTRL_H211B && !o->replay_dt) {
            // Eqs. 51-54 (see the oracle's controller for the reading of Fig. 5)
            lim = 0.0;
            double err = INFINITY;
            int tries = 0;
            bool aborted = false;
            while (err > 1.02 * o->tol || lim < 0.9) {
                out->attempts++;
                dg_status sC = attempt_(ctx, cur, ctx->zC, t, dt, &info);
                dg_status sF1 = sC == DG_OK ? attempt_(ctx, cur, nxt, t, 0.5 * dt, &info) : sC;
                dg_status sF = sF1 == DG_OK ? attempt_(ctx, nxt, ctx->zF, t + 0.5 * dt, 0.5 * dt, &info) : sF1;
                if (sF != DG_OK && sF != DG_ERR_NOCONV && sF != DG_ERR_NONFINITE) return sF;
                if (sF != DG_OK) {
                    out->failures++;
                    dt *= 0.5;
                    ++halv;
                    lim = 0.0;
                    err = INFINITY;
                    if (halv > max_h || dt < o->dt_min) { aborted = true; break; }
                    continue;
                }
                halv = 0;
                dg_status se;
                err = std::max(rel_err_(ctx, ctx->zF, ctx->zC, &se), 1e-300);
                if (se != DG_OK) return se;
                double ratio = std::pow(o->tol / err, 0.25) * std::pow(o->tol / err_prev, 0.25) * std::pow(dt / dt_prev, -0.25);
                lim = 1.0 + std::atan(ratio - 1.0);
                if (err > 1.02 * o->tol || lim < 0.9) {
                    if (++tries > 50) { aborted = true; break; }
                    err_prev = err;
                    dt_prev = dt;
                    dt = std::min(dt * lim, o->dt_max);
                }
            }
            if (aborted) { result = fail(ctx, DG_ERR_ABORTED, "H211b controller gave up"); break; }
            // Richardson extrapolation, Eq. 54: z = 2 z_F - z_C
            CK(cudaMemcpyAsync(nxt, ctx->zF, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
            CK(axpby(L, nxt, 2.0, ctx->zC, -1.0, N));
            err_prev = err;
            dt_prev = dt;
            ok = true;
        } else {
            out->attempts++;
            dg_status s = attempt_(ctx, cur, nxt, t, dt, &info);
            if (s != DG_OK && s != DG_ERR_NOCONV && s != DG_ERR_NONFINITE) return s;
            ok = s == DG_OK;
        }
        if (ok) {
            std::swap(cur, nxt);
            t += dt;
            halv = 0;
            if (o->limiter && ctx->P.order == 1) CK(dg1_limit(L, ctx->P, ctx->G, cur, ctx->gbd));
            double U;
            dg_status s = dg_cell_voltage(ctx, cur, &U);
            if (s != DG_OK) return s;
            out->t[n] = t;
            out->dt[n] = dt;
            out->U_cell[n] = U;
            out->c_m[n] = t / 3600.0 * ctx->prm.f_C * c_theo_ah;
            if (out->newton_its) out->newton_its[n] = info.newton_iterations;
            if (out->gmres_its) out->gmres_its[n] = info.gmres_iterations;
            ++n;
            out->n = n;
            if (U <= o->cutoff_V) break;
            if (o->controller == DG_CTRL_H211B && !o->replay_dt) {
                dt = std::min(lim * dt, o->dt_max);
            } else if (o->controller == DG_CTRL_NAIVE && !o->replay_dt) {
                if (++sct == 3) { dt *= 1.2; sct = 0; }
                dt = std::min(dt, o->dt_max);
            }
        } else {
            if (o->replay_dt) { result = fail(ctx, DG_ERR_NOCONV, "replayed step did not converge"); break; }
            out->failures++;
            dt *= 0.5;
            sct = 0;
            if (++halv > max_h || dt < o->dt_min) { result = fail(ctx, DG_ERR_ABORTED, "30 consecutive halvings"); break; }
        }
    }
    CK(cudaMemcpyAsync(z, cur, N * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    dg_status s = sync_(ctx);
    out->status = result;
    if (out->checkpoint) {
        out->checkpoint->t = t;
        out->checkpoint->dt = dt;
        out->checkpoint->err_prev = err_prev;
        out->checkpoint->dt_prev = dt_prev;
        out->checkpoint->sct = sct;
        out->checkpoint->halvings = halv;
    }
    return result != DG_OK ? result : s;
}

// ------------------------------------------------------------------ allocation-free residual
// For callers that must not allocate device memory at the time of the call -- code running
// inside CUDA stream capture (cudaMalloc is not allowed there) or under an external allocator
// that owns all device memory -- and that must not touch the context's own workspaces: the
// DG0 residual with its transport-factor scratch in a static device array instead of the
// context's buffer.  The array is part of the library image, so every GPU that loads the
// library holds it (NOALLOC_MAX_VOXELS doubles = 16 MiB) until the process exits.
namespace {
constexpr int64_t NOALLOC_MAX_VOXELS = 2097152;   // 128^3 voxels
__device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_VOXELS];
constexpr int NOALLOC_MAX_DEVICES = 64;
// device address of the array per device, looked up once; atomic because several host threads
// (one per serving slot) may make their first call on a device at the same time
std::atomic<double*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" dg_status dg_residual_noalloc(dg_ctx* ctx, const double* z, const double* zold, double t, double dt,
                                         double* r) {
    if (!ctx || !z || !zold || !r || !(dt > 0)) return fail(ctx, DG_ERR_ARG, "dg_residual_noalloc: bad argument");
    if (ctx->P.order != 0)
        return fail(ctx, DG_ERR_ARG, "dg_residual_noalloc: DG0 contexts only (DG1 needs 32 scratch values per voxel)");
    if ((int64_t)ctx->P.n_cell > NOALLOC_MAX_VOXELS)
        return fail(ctx, DG_ERR_ARG, "dg_residual_noalloc: " + std::to_string(ctx->P.n_cell) +
                                         " voxels exceed the static scratch of " + std::to_string(NOALLOC_MAX_VOXELS));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(ctx, DG_ERR_ARG, "dg_residual_noalloc: device index too large");
    double* scratch = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        // once per device, with that device current: the host-side name of a __device__ array is
        // not a device address, so ask the runtime for it (two racing first calls store the same value)
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        scratch = (double*)ptr;
        g_noalloc_ptr[dev].store(scratch, std::memory_order_release);
    }
    int64_t launches = 0;
    LaunchCtx L{ctx->L.st, &launches};
    e = dg0_residual(L, ctx->P, ctx->G, z, zold, t, dt, 0, r, scratch);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_residual_noalloc: ") + cudaGetErrorString(e));
    return DG_OK;
}

// ------------------------------------------------------------------ batches of instances
// Several contexts (uneven grids, either DG order, one chemistry) evaluated together: the fused
// DG1 product, the DG0 product and the DG0 residual of all instances each run as one launch over
// the instances' concatenated blocks (job records in device memory, block -> (instance, block)
// maps as the schedule); implicit steps of all instances run concurrently, each on its own
// context's stream.
struct dg_batch {
    std::vector<dg_ctx*> ctx;
    LaunchCtx L{};
    int64_t launches = 0;
    std::string err;
    bool tradeoff = true;
    std::vector<int> k0, k1;                       // instances of order 0 and 1
    static constexpr int N_SCHED1 = 2, N_BS0 = 4;  // DG1 block orders; DG0 block sizes
    int2* d_map1[N_SCHED1] = {};
    int nblk1 = 0;
    int2* d_map0[N_BS0] = {};
    int nblk0[N_BS0] = {};
    int bs0[N_BS0] = {64, 128, 256, 512};
    int2* d_mapc = nullptr;                        // FP32 conversion of every instance's z
    int nblkc = 0;
    int sched1 = 0, sched0 = 1;                    // schedules in use (dg_batch_autotune chooses)
    size_t sz1 = 0;                                // bytes of one DG1 job record (the larger precision)
    unsigned char *d_job1 = nullptr, *h_job1 = nullptr;
    Job0<double>* d_job0 = nullptr;                // Job0<float> has the same size (pointers, doubles)
    Job0<double>* h_job0 = nullptr;
    ConvJob *d_conv = nullptr, *h_conv = nullptr;
    cudaEvent_t staged = nullptr;                  // the device has read the staging buffers
    std::vector<void*> dev, host;
};

// the host writes FP32 and FP64 DG0 job records into one array: they must have the same size
static_assert(sizeof(Job0<float>) == sizeof(Job0<double>), "DG0 job records of both precisions");

static dg_status bfail(dg_batch* b, dg_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}
#define BCK(x)                                                                                        \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) return bfail(b, DG_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void batch_free(dg_batch* b) {
    for (void* p : b->dev) cudaFree(p);
    for (void* p : b->host) cudaFreeHost(p);
    if (b->staged) cudaEventDestroy(b->staged);
    b->dev.clear();
    b->host.clear();
}

// block -> (instance, block) maps: instance after instance, or one block of each instance in turn
static std::vector<int2> batch_map(const std::vector<int64_t>& nb, bool round_robin) {
    std::vector<int2> m;
    if (!round_robin) {
        for (size_t j = 0; j < nb.size(); ++j)
            for (int64_t q = 0; q < nb[j]; ++q) m.push_back(make_int2((int)j, (int)q));
        return m;
    }
    int64_t most = 0;
    for (int64_t x : nb) most = std::max(most, x);
    for (int64_t q = 0; q < most; ++q)
        for (size_t j = 0; j < nb.size(); ++j)
            if (q < nb[j]) m.push_back(make_int2((int)j, (int)q));
    return m;
}

extern "C" dg_status dg_batch_create(dg_ctx* const* ctxs, int32_t n, void* stream, dg_batch** out) {
    if (!out) return DG_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n < 1) return DG_ERR_ARG;
    dg_batch* b = new dg_batch;
    b->L.st = (cudaStream_t)stream;
    b->L.counter = &b->launches;
    for (int k = 0; k < n; ++k) {
        if (!ctxs[k]) { delete b; return DG_ERR_ARG; }
        b->ctx.push_back(ctxs[k]);
        (ctxs[k]->P.order == 1 ? b->k1 : b->k0).push_back(k);
    }
    b->tradeoff = ctxs[0]->P.nf == 10;
    for (dg_ctx* c : b->ctx)
        if ((c->P.nf == 10) != b->tradeoff) { delete b; return DG_ERR_ARG; }   // one chemistry per batch
    auto upload = [&](const std::vector<int2>& m, int2** d) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(1, m.size()) * sizeof(int2));
        if (e != cudaSuccess) return e;
        b->dev.push_back(*d);
        return m.empty() ? cudaSuccess : cudaMemcpy(*d, m.data(), m.size() * sizeof(int2), cudaMemcpyHostToDevice);
    };
    cudaError_t e = cudaSuccess;
    std::vector<int64_t> nb1;
    for (int k : b->k1) nb1.push_back((b->ctx[k]->P.n_cell + FUSED_VOXELS - 1) / FUSED_VOXELS);
    for (int s = 0; s < dg_batch::N_SCHED1 && e == cudaSuccess; ++s) {
        std::vector<int2> m = batch_map(nb1, s == 1);
        b->nblk1 = (int)m.size();
        e = upload(m, &b->d_map1[s]);
    }
    for (int q = 0; q < dg_batch::N_BS0 && e == cudaSuccess; ++q) {
        std::vector<int64_t> nb0;
        for (int k : b->k0) nb0.push_back((b->ctx[k]->P.n_cell + b->bs0[q] - 1) / b->bs0[q]);
        std::vector<int2> m = batch_map(nb0, false);
        b->nblk0[q] = (int)m.size();
        e = upload(m, &b->d_map0[q]);
    }
    if (e == cudaSuccess) {
        std::vector<int64_t> nbc;
        for (dg_ctx* c : b->ctx) nbc.push_back((c->ndof + CONV_BLOCK_ELEMS - 1) / CONV_BLOCK_ELEMS);
        std::vector<int2> m = batch_map(nbc, false);
        b->nblkc = (int)m.size();
        e = upload(m, &b->d_mapc);
    }
    b->sz1 = std::max(dg1_job_bytes(false), dg1_job_bytes(true));
    auto dal = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (r == cudaSuccess) b->dev.push_back(*p);
        return r;
    };
    auto hal = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMallocHost(p, std::max<size_t>(bytes, 16));
        if (r == cudaSuccess) b->host.push_back(*p);
        return r;
    };
    if (e == cudaSuccess) e = dal((void**)&b->d_job1, n * b->sz1);
    if (e == cudaSuccess) e = hal((void**)&b->h_job1, n * b->sz1);
    if (e == cudaSuccess) e = dal((void**)&b->d_job0, n * sizeof(Job0<double>));
    if (e == cudaSuccess) e = hal((void**)&b->h_job0, n * sizeof(Job0<double>));
    if (e == cudaSuccess) e = dal((void**)&b->d_conv, n * sizeof(ConvJob));
    if (e == cudaSuccess) e = hal((void**)&b->h_conv, n * sizeof(ConvJob));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess && b->staged) e = cudaEventRecord(b->staged, b->L.st);
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return DG_ERR_CUDA;
    }
    *out = b;
    return DG_OK;
}

extern "C" dg_status dg_batch_destroy(dg_batch* b) {
    if (!b) return DG_ERR_ARG;
    cudaStreamSynchronize(b->L.st);
    batch_free(b);
    delete b;
    return DG_OK;
}

extern "C" const char* dg_batch_last_error(const dg_batch* b) { return b ? b->err.c_str() : "null batch"; }
extern "C" int64_t dg_batch_launch_count(const dg_batch* b) { return b ? b->launches : 0; }

// the staging buffers may be rewritten once the device has read the previous upload
static dg_status batch_stage_wait(dg_batch* b) {
    BCK(cudaEventSynchronize(b->staged));
    return DG_OK;
}

static dg_status batch_upload(dg_batch* b, bool j1, bool j0, bool conv) {
    const int n = (int)b->ctx.size();
    if (j1) BCK(cudaMemcpyAsync(b->d_job1, b->h_job1, n * b->sz1, cudaMemcpyHostToDevice, b->L.st));
    if (j0) BCK(cudaMemcpyAsync(b->d_job0, b->h_job0, n * sizeof(Job0<double>), cudaMemcpyHostToDevice, b->L.st));
    if (conv) BCK(cudaMemcpyAsync(b->d_conv, b->h_conv, n * sizeof(ConvJob), cudaMemcpyHostToDevice, b->L.st));
    BCK(cudaEventRecord(b->staged, b->L.st));
    return DG_OK;
}

template <class S>
static void job0_fill(dg_ctx* c, const S* z, const S* v, const double* zn, double t, double dt, S* out, Job0<S>* J) {
    std::memset((void*)J, 0, sizeof(*J));
    J->p = c->P;
    J->g = c->G;
    J->z = z;
    J->v = v;
    J->zn = zn;
    const bool f32 = std::is_same<S, float>::value;
    J->gb = f32 ? (S*)c->gb32 : (S*)c->gb;
    J->gbd = f32 ? (S*)c->gbd32 : (S*)c->gbd;
    J->out = out;
    J->t = t;
    J->dt = dt;
    J->sc_dt = 0.0;
    J->relax = 0;
}

// launch the products of all instances (the jobs are uploaded; sched: schedules to use)
static dg_status batch_jvp_launch(dg_batch* b, bool f32, int s1, int s0) {
    if (f32) BCK(to_f32_batched(b->L, b->d_conv, b->d_mapc, b->nblkc));
    BCK(dg1_jvp_fused_batched(b->L, f32, b->tradeoff, b->d_job1, b->d_map1[s1], b->k1.empty() ? 0 : b->nblk1));
    if (f32) BCK(dg0_batch<float>(b->L, b->tradeoff, 1, (const Job0<float>*)b->d_job0, b->d_map0[s0], b->nblk0[s0], b->bs0[s0]));
    else BCK(dg0_batch<double>(b->L, b->tradeoff, 1, b->d_job0, b->d_map0[s0], b->nblk0[s0], b->bs0[s0]));
    return DG_OK;
}

static dg_status batch_jvp_stage(dg_batch* b, const double* const* z, const double* t, const double* dt,
                                 int32_t precision, const void* const* v, void* const* jv) {
    if (!z || !t || !dt || !v || !jv) return bfail(b, DG_ERR_ARG, "dg_batch_jvp: bad argument");
    const bool f32 = precision == DG_PREC_MIXED;
    if (!f32 && precision != DG_PREC_FP64) return bfail(b, DG_ERR_ARG, "dg_batch_jvp: precision must be FP64 or MIXED");
    for (size_t k = 0; k < b->ctx.size(); ++k) {
        if (!z[k] || !v[k] || !jv[k] || !(dt[k] > 0)) return bfail(b, DG_ERR_ARG, "dg_batch_jvp: bad instance argument");
        if (f32 && (b->ctx[k]->prm.precision != DG_PREC_MIXED || !b->ctx[k]->z32))
            return bfail(b, DG_ERR_ARG, "dg_batch_jvp: FP32 products need contexts set up with DG_PREC_MIXED");
    }
    dg_status s = batch_stage_wait(b);
    if (s != DG_OK) return s;
    const size_t sz = dg1_job_bytes(f32);          // the kernel of this precision indexes records at its size
    for (size_t j = 0; j < b->k1.size(); ++j) {
        dg_ctx* c = b->ctx[b->k1[j]];
        const int k = b->k1[j];
        const void* zz = f32 ? (const void*)c->z32 : (const void*)z[k];
        dg1_fused_job(f32, c->P, c->G, zz, v[k], t[k], dt[k], 0, 0.0, jv[k], b->h_job1 + j * sz);
    }
    for (size_t j = 0; j < b->k0.size(); ++j) {
        const int k = b->k0[j];
        dg_ctx* c = b->ctx[k];
        if (f32) job0_fill<float>(c, c->z32, (const float*)v[k], nullptr, t[k], dt[k], (float*)jv[k], (Job0<float>*)(b->h_job0 + j));
        else job0_fill<double>(c, z[k], (const double*)v[k], nullptr, t[k], dt[k], (double*)jv[k], b->h_job0 + j);
    }
    for (size_t k = 0; k < b->ctx.size(); ++k) b->h_conv[k] = ConvJob{z[k], b->ctx[k]->z32, b->ctx[k]->ndof};
    return batch_upload(b, true, true, f32);
}

extern "C" dg_status dg_batch_jvp(dg_batch* b, const double* const* z, const double* t, const double* dt,
                                  int32_t precision, const void* const* v, void* const* jv) {
    if (!b) return DG_ERR_ARG;
    dg_status s = batch_jvp_stage(b, z, t, dt, precision, v, jv);
    if (s != DG_OK) return s;
    return batch_jvp_launch(b, precision == DG_PREC_MIXED, b->sched1, b->sched0);
}

extern "C" dg_status dg_batch_residual(dg_batch* b, const double* const* z, const double* const* zold,
                                       const double* t, const double* dt, double* const* r) {
    if (!b) return DG_ERR_ARG;
    if (!z || !zold || !t || !dt || !r) return bfail(b, DG_ERR_ARG, "dg_batch_residual: bad argument");
    for (size_t k = 0; k < b->ctx.size(); ++k)
        if (!z[k] || !zold[k] || !r[k] || !(dt[k] > 0)) return bfail(b, DG_ERR_ARG, "dg_batch_residual: bad instance argument");
    dg_status s = batch_stage_wait(b);
    if (s != DG_OK) return s;
    for (size_t j = 0; j < b->k0.size(); ++j) {
        const int k = b->k0[j];
        job0_fill<double>(b->ctx[k], z[k], z[k], zold[k], t[k], dt[k], r[k], b->h_job0 + j);
    }
    s = batch_upload(b, false, true, false);
    if (s != DG_OK) return s;
    // 128-voxel blocks, the block size of the single-instance residual kernels
    BCK(dg0_batch<double>(b->L, b->tradeoff, 0, b->d_job0, b->d_map0[1], b->nblk0[1], b->bs0[1]));
    // DG1 residuals: the instances' own face-once kernels, issued on the batch stream
    for (int k : b->k1) {
        dg_ctx* c = b->ctx[k];
        BCK(dg1_residual(b->L, c->P, c->G, z[k], zold[k], t[k], dt[k], 0, r[k], c->gb, c->gbd));
    }
    return DG_OK;
}

extern "C" dg_status dg_batch_autotune(dg_batch* b, const double* const* z, const double* t, const double* dt,
                                       int32_t precision, const void* const* v, void* const* jv, int32_t choice[2]) {
    if (!b) return DG_ERR_ARG;
    dg_status s = batch_jvp_stage(b, z, t, dt, precision, v, jv);
    if (s != DG_OK) return s;
    const bool f32 = precision == DG_PREC_MIXED;
    if (f32) BCK(to_f32_batched(b->L, b->d_conv, b->d_mapc, b->nblkc));
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    auto timed = [&](auto launch) -> double {
        launch();                                   // warm-up
        cudaEventRecord(e0, b->L.st);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1, b->L.st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // a candidate whose launches fail is not a candidate (its time would be that of doing nothing)
    cudaError_t trial = cudaSuccess;
    double best = 1e30;
    if (!b->k1.empty()) {
        for (int q = 0; q < dg_batch::N_SCHED1; ++q) {
            trial = cudaSuccess;
            double ms = timed([&] {
                cudaError_t r = dg1_jvp_fused_batched(b->L, f32, b->tradeoff, b->d_job1, b->d_map1[q], b->nblk1);
                if (r != cudaSuccess) trial = r;
            });
            if (trial == cudaSuccess && ms < best) { best = ms; b->sched1 = q; }
        }
    }
    best = 1e30;
    if (!b->k0.empty()) {
        const int maxbs = dg0_batch_max_block(b->tradeoff, f32);
        for (int q = 0; q < dg_batch::N_BS0; ++q) {
            if (b->bs0[q] > maxbs) continue;
            trial = cudaSuccess;
            double ms = timed([&] {
                cudaError_t r = f32 ? dg0_batch<float>(b->L, b->tradeoff, 1, (const Job0<float>*)b->d_job0, b->d_map0[q],
                                                       b->nblk0[q], b->bs0[q])
                                    : dg0_batch<double>(b->L, b->tradeoff, 1, b->d_job0, b->d_map0[q], b->nblk0[q], b->bs0[q]);
                if (r != cudaSuccess) trial = r;
            });
            if (trial == cudaSuccess && ms < best) { best = ms; b->sched0 = q; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaGetLastError());
    if (choice) { choice[0] = b->sched1; choice[1] = b->bs0[b->sched0]; }
    return DG_OK;
}

extern "C" dg_status dg_batch_step(dg_batch* b, const double* const* zn, double* const* z, const double* t,
                                   const double* dt, dg_step_info* info, int32_t* status) {
    if (!b || !zn || !z || !t || !dt || !status) return bfail(b, DG_ERR_ARG, "dg_batch_step: bad argument");
    const size_t n = b->ctx.size();
    std::vector<std::thread> th;
    for (size_t k = 0; k < n; ++k)
        th.emplace_back([&, k] { status[k] = dg_step(b->ctx[k], zn[k], z[k], t[k], dt[k], info ? info + k : nullptr); });
    for (auto& x : th) x.join();
    return DG_OK;
}
