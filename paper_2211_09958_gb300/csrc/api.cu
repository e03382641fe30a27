// C ABI of the GB300 PM library: context, cuFFT plans and the pipelines
// (force, KDK step, integration, reverse-time adjoint, initial conditions,
// density, power spectrum).  See include/pmgb.h for the contract.

#include <cufft.h>

#include <cmath>
#include <functional>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pmgb.h"
#include "pm_internal.h"

using namespace pmgb;

namespace {

constexpr int kMeshFields = 4;   // scratch meshes: density/force (0..2), adjoint psi (3)
constexpr int kLatFields = 14;   // IC lattice fields (see pm_init_lpt_adjoint)

thread_local std::string g_create_error;

}  // namespace

struct pm_ctx {
    Params P;
    std::vector<double> om, s8;
    std::vector<HostTables> tabs;
    int device = 0;
    cudaStream_t stream = nullptr;
    Geom g{};
    int64_t mesh_pad = 0;  // floats of one padded n_m^3 field
    int64_t lat_pad = 0;   // floats of one padded n_p^3 field
    float *mesh = nullptr;
    float *lat = nullptr;
    float4 *d_table = nullptr;
    float *d_pref = nullptr;
    float *d_grad = nullptr;  // [n_m] difference-gradient multiplier per axis index
    float *d_dec = nullptr;   // [n_m] CIC deconvolution factor per axis index (solver flag)
    float4 *d_fac = nullptr;
    LinParams *d_lin = nullptr;
    double *d_red = nullptr;
    double *d_pk = nullptr;
    double *d_lred = nullptr;
    cufftHandle r2c = 0, c2r = 0, lr2c = 0, lc2r = 0;
    // own FFT (power-of-two meshes): real meshes r1 ([run][n^3]) and r4
    // ([run][n^3][4] interleaved), four spectrum fields, twiddle table
    bool own = false;
    FftGeom fg{};
    float *r1 = nullptr, *r4 = nullptr;
    float *rpot = nullptr;   // [run][n^3][2]: potential phi (and adjoint psi) before the gradient stencil
    float2 *spec = nullptr, *tw = nullptr;
    ZInvMap zmaps[Z_INV_MAPS] = {};  // TMA descriptors of the blocked spectrum (z inverse)
    int *d_err = nullptr;    // device error flag (bounded TMA waits)
    bool have_plans = false;
    void *work = nullptr;
    std::string err;
    int64_t launches = 0;
    // kernel timing (pm_profile): event pairs per launch, grouped by kind
    bool prof = false;
    std::vector<std::string> kinds;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<int> rec_kind;
    // CUDA graphs of the integration loops, replayed when a call repeats
    // with the same steps and buffers
    bool graphs_on = true;
    cudaStream_t cap_stream = nullptr;
    struct GraphEntry {
        int kind, b, e;
        const void *q[5];
        uint32_t flags;
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::vector<GraphEntry> graphs;
    // sparse checkpoints (pm_set_checkpoints): s_m and p_{m+1/2} of the last
    // forward run at steps m = every, 2 every, ... in a caller-owned buffer
    int ck_every = 0;
    float *ck_buf = nullptr;
    // launch shapes of the tunable kernel families: block sizes of paint,
    // read, spectral force/adjoint, z-pass FFT (n >= 256); x-pass pencil width
    // shape; z-inverse and z-forward staging; x round trip; force pipeline
    int tune[PM_TUNE_KINDS] = {256, 256, 256, 256, 8, 2, 1, 2, 2, 1};
    // binned tile-owned deposit (own-FFT meshes, CIC, n_m a multiple of 16;
    // dep_ok: supported here): bin keys, ranks and CSR of the particles,
    // counters, scan scratch, halo lines, allocated when it is first selected
    bool dep_ok = false;
    // r1 / r4 known to hold zeros (cleared by the previous read of the same
    // integration call), so that the next paint can skip its zeroing pass;
    // false outside the integration loops
    bool r1_zero = false, r4_zero = false;
    int *dep_key = nullptr, *dep_rank = nullptr, *dep_idx = nullptr, *dep_count = nullptr, *dep_offset = nullptr,
        *dep_chunk = nullptr;
    float *dep_halo = nullptr;
    // learned force correction (own-FFT meshes only)
    bool nn_on = false;
    void *nn_packed = nullptr;
    NNWeightsMut nnw{};
    float *nn_theta = nullptr, *nn_grad = nullptr, *nn_m = nullptr, *nn_v = nullptr, *nn_part = nullptr;
    __nv_bfloat16 *nn_act = nullptr;
    double *nn_loss = nullptr;
    int *nn_err = nullptr;  // tensor-core kernel time-out flag
    __nv_bfloat16 *nn_feat = nullptr;  // feature mesh [run][n^3]
    float *nn_mesh4 = nullptr;         // [run][n^3][4]: correction (0..2) and density cotangent (3) of an adjoint step
    float *nn_gx = nullptr;            // [cells][32] feature cotangents
};

namespace {

int fail(pm_ctx *ctx, int code, const std::string &msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return code;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int kind_id(pm_ctx *ctx, const char *name) {
    for (size_t i = 0; i < ctx->kinds.size(); ++i)
        if (ctx->kinds[i] == name) return (int)i;
    ctx->kinds.emplace_back(name);
    return (int)ctx->kinds.size() - 1;
}

cudaEvent_t pool_event(pm_ctx *ctx) {
    if (ctx->pool_used == ctx->pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->pool.push_back(e);
    }
    return ctx->pool[ctx->pool_used++];
}

// Records an event pair around one launch on the context stream when
// profiling is on; a failure to get events only drops that record.
struct ProfScope {
    pm_ctx *ctx;
    const char *kind;
    cudaEvent_t a = nullptr;
    ProfScope(pm_ctx *c, const char *k) : ctx(c), kind(k) {
        if (ctx->prof && (a = pool_event(ctx)) != nullptr) cudaEventRecord(a, ctx->stream);
    }
    void end() {
        if (!a) return;
        cudaEvent_t b = pool_event(ctx);
        if (!b) {
            ctx->pool_used--;
            a = nullptr;
            return;
        }
        cudaEventRecord(b, ctx->stream);
        ctx->rec_kind.push_back(kind_id(ctx, kind));
        a = nullptr;
    }
};

const char *paint_kind(int mode) { return mode == PAINT_ADJ ? "paint_adj" : "paint_density"; }

const char *read_kind(int mode) {
    switch (mode) {
        case READ_FORCE: return "read_force";
        case READ_KICK_DRIFT: return "read_kick_drift";
        case READ_HALF_KICK: return "read_half_kick";
        case READ_ADJ: return "read_adj";
        default: return "read_grad";
    }
}

#define PM_CUDA(ctx, x)                                                                                   \
    do {                                                                                                  \
        cudaError_t e_ = (x);                                                                             \
        if (e_ != cudaSuccess) return fail(ctx, PM_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define PM_LAUNCH(ctx, kind, x)                                                                           \
    do {                                                                                                  \
        ProfScope ps_(ctx, kind);                                                                         \
        cudaError_t e_ = (x);                                                                             \
        ps_.end();                                                                                        \
        (ctx)->launches++;                                                                                \
        if (e_ != cudaSuccess) return fail(ctx, PM_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define PM_MEMSET(ctx, x)                                                                                 \
    do {                                                                                                  \
        ProfScope ps_(ctx, "memset");                                                                     \
        cudaError_t e_ = (x);                                                                             \
        ps_.end();                                                                                        \
        if (e_ != cudaSuccess) return fail(ctx, PM_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define PM_FFT(ctx, x)                                                                     \
    do {                                                                                   \
        cufftResult r_ = (x);                                                              \
        if (r_ != CUFFT_SUCCESS)                                                           \
            return fail(ctx, PM_ECUFFT, std::string(#x ": cufft error ") + std::to_string((int)r_)); \
    } while (0)

#define PM_TRY(x)              \
    do {                       \
        int rc_ = (x);         \
        if (rc_ != PM_OK) return rc_; \
    } while (0)

int64_t padded(int n) { return (int64_t)n * n * 2 * (n / 2 + 1); }

int make_plan(pm_ctx *ctx, cufftHandle *h, int n, bool r2c, long long batch, size_t *ws) {
    PM_FFT(ctx, cufftCreate(h));
    PM_FFT(ctx, cufftSetAutoAllocation(*h, 0));
    long long dims[3] = {n, n, n};
    long long rembed[3] = {n, n, 2LL * (n / 2 + 1)};
    long long cembed[3] = {n, n, n / 2 + 1};
    const long long rdist = (long long)n * n * 2 * (n / 2 + 1);
    const long long cdist = (long long)n * n * (n / 2 + 1);
    if (r2c)
        PM_FFT(ctx, cufftMakePlanMany64(*h, 3, dims, rembed, 1, rdist, cembed, 1, cdist, CUFFT_R2C, batch, ws));
    else
        PM_FFT(ctx, cufftMakePlanMany64(*h, 3, dims, cembed, 1, cdist, rembed, 1, rdist, CUFFT_C2R, batch, ws));
    return PM_OK;
}

int upload_tables(pm_ctx *ctx) {
    const int B = ctx->P.n_batch, N = ctx->P.n_steps;
    ctx->tabs.resize(B);
    for (int b = 0; b < B; ++b) host_tables(ctx->P, ctx->om[b], ctx->s8[b], &ctx->tabs[b]);
    std::vector<float4> table((size_t)N * B);
    std::vector<float> pref(B);
    std::vector<float4> fac(B);
    std::vector<LinParams> lin(B);
    const double n3 = (double)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    const double vc = std::pow(ctx->P.box / ctx->P.n_p, 3);
    for (int b = 0; b < B; ++b) {
        const HostTables &t = ctx->tabs[b];
        for (int n = 0; n < N; ++n) {
            const double merged = t.ka[n] + (n > 0 ? t.kb[n - 1] : 0.0);
            table[(size_t)n * B + b] = make_float4((float)t.ka[n], (float)t.dr[n], (float)t.kb[n], (float)merged);
        }
        pref[b] = (float)(1.5 * ctx->om[b] / n3);
        fac[b] = make_float4((float)t.lpt[0], (float)t.lpt[1], (float)t.lpt[2], (float)t.lpt[3]);
        lin[b] = LinParams{t.amp, ctx->om[b], ctx->P.h, ctx->P.n_s, t.dlnamp, 1.0 / vc};
    }
    PM_CUDA(ctx, cudaMemcpy(ctx->d_table, table.data(), sizeof(float4) * table.size(), cudaMemcpyHostToDevice));
    PM_CUDA(ctx, cudaMemcpy(ctx->d_pref, pref.data(), sizeof(float) * B, cudaMemcpyHostToDevice));
    PM_CUDA(ctx, cudaMemcpy(ctx->d_fac, fac.data(), sizeof(float4) * B, cudaMemcpyHostToDevice));
    PM_CUDA(ctx, cudaMemcpy(ctx->d_lin, lin.data(), sizeof(LinParams) * B, cudaMemcpyHostToDevice));
    return PM_OK;
}

int check_cosmology(pm_ctx *ctx, const double *om, const double *s8, int B, int solver = 0) {
    if (!om || !s8) return fail(ctx, PM_EINVAL, "omega_m and sigma8 must be host arrays of n_batch values");
    for (int b = 0; b < B; ++b) {
        if (!(om[b] > 0.0 && om[b] <= 1.0)) return fail(ctx, PM_EINVAL, "omega_m must be in (0, 1]");
        if (!(s8[b] > 0.0)) return fail(ctx, PM_EINVAL, "sigma8 must be > 0");
        if ((solver & PM_SOLVER_GROWTH_EMULATOR) && !growth_emulator_covers(om[b], 0.5))
            return fail(ctx, PM_ERANGE, "the growth emulator covers omega_m in [0.1, 0.6]");
    }
    return PM_OK;
}

// The time range the growth emulator covers (solver flag 16).
int check_emulator_range(double a_init, double a_final, int solver) {
    if ((solver & PM_SOLVER_GROWTH_EMULATOR) &&
        !(growth_emulator_covers(0.3, a_init) && growth_emulator_covers(0.3, a_final)))
        return fail(nullptr, PM_ERANGE, "the growth emulator covers a in [1e-3, 1]");
    return PM_OK;
}

// --------------------------------------------------------------- pieces --

// The force meshes the read kernels interpolate from.
MeshRef mesh_ref(pm_ctx *ctx) {
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    if (ctx->own) return MeshRef{ctx->r4, 0, 4 * n3, ctx->P.n_m, 4};
    return MeshRef{ctx->mesh, ctx->mesh_pad * ctx->P.n_batch, ctx->mesh_pad, 2 * (ctx->P.n_m / 2 + 1), 0};
}

// A single real scratch field (density).
MeshRef density_ref(pm_ctx *ctx) {
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    if (ctx->own) return MeshRef{ctx->r1, 0, n3, ctx->P.n_m, 0};
    return MeshRef{ctx->mesh, 0, ctx->mesh_pad, 2 * (ctx->P.n_m / 2 + 1), 0};
}

int64_t density_floats(pm_ctx *ctx) {
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    return (ctx->own ? n3 : ctx->mesh_pad) * ctx->P.n_batch;
}

Spec mesh_spec(pm_ctx *ctx) {
    const float kf = (float)(2.0 * M_PI / ctx->P.box);
    const int n = ctx->P.n_m;
    if (ctx->own) {
        const int64_t per = (int64_t)n * n * ctx->fg.zc;
        return Spec{ctx->spec, per * ctx->P.n_batch, per, n, ctx->P.n_batch, kf, ctx->fg.zc, 1, ctx->d_grad,
                    ctx->d_dec, ctx->tune[2]};
    }
    const int64_t modes = ctx->mesh_pad / 2;
    return Spec{reinterpret_cast<float2 *>(ctx->mesh), modes * ctx->P.n_batch, modes, n, ctx->P.n_batch, kf, n / 2 + 1, 0,
                ctx->d_grad, ctx->d_dec, ctx->tune[2]};
}

// Whether a force (adj = false) or adjoint evaluation takes the fused x
// round trip: x_round tuning 2 = both, 3 = the force only.
bool x_fused(const pm_ctx *ctx, bool adj) { return ctx->tune[7] == 2 || (ctx->tune[7] == 3 && !adj); }

// Whether force evaluations take the potential pipeline (tuning family 8 =
// 2): one inverse transform of phi = IFFT(g delta) (and psi for the adjoint)
// and the 4-point difference F_j = S_j phi on the real mesh, instead of three
// inverse transforms of i D_j g delta.  The two are the same linear map; the
// stencil form exists only for the 4-point difference gradient.
bool pot_pipeline(const pm_ctx *ctx) {
    return ctx->own && ctx->tune[8] == 2 && !(ctx->P.solver & PM_SOLVER_SPECTRAL_GRADIENT);
}

// Whether the CIC read takes the force straight from the potential mesh (the
// difference formed per corner in the read kernel) instead of from the float4
// force mesh of the stencil pass: the potential pipeline with CIC assignment
// and without the learned correction (which adds to the force mesh).
bool pot_read(const pm_ctx *ctx) { return pot_pipeline(ctx) && ctx->g.order == 2 && !ctx->nn_on; }

// Multipliers of the fused x round trip: the spectral kernels' tables.
XRoundArgs xround_args(pm_ctx *ctx) {
    return XRoundArgs{(float)(2.0 * M_PI / ctx->P.box), ctx->d_grad, ctx->d_dec, ctx->d_pref,
                      (float)(ctx->P.n_m / (12.0 * ctx->P.box)), (ctx->P.solver & PM_SOLVER_SPECTRAL_GRADIENT) ? 0 : 1};
}

MeshRef lat_ref(pm_ctx *ctx) {
    return MeshRef{ctx->lat, ctx->lat_pad * ctx->P.n_batch, ctx->lat_pad, 2 * (ctx->P.n_p / 2 + 1), 0};
}

Spec lat_spec(pm_ctx *ctx) {
    const int64_t modes = ctx->lat_pad / 2;
    return Spec{reinterpret_cast<float2 *>(ctx->lat), modes * ctx->P.n_batch, modes, ctx->P.n_p, ctx->P.n_batch,
                (float)(2.0 * M_PI / ctx->P.box), ctx->P.n_p / 2 + 1, 0};
}

float *lat_field(pm_ctx *ctx, int f) { return ctx->lat + (int64_t)f * ctx->lat_pad * ctx->P.n_batch; }

int fft_fields(pm_ctx *ctx, cufftHandle plan, bool r2c, float *base, int64_t fstride, int f0, int nf) {
    for (int f = f0; f < f0 + nf; ++f) {
        float *p = base + (int64_t)f * fstride;
        ProfScope ps(ctx, r2c ? "cufft_r2c" : "cufft_c2r");
        const cufftResult r = r2c ? cufftExecR2C(plan, p, reinterpret_cast<cufftComplex *>(p))
                                  : cufftExecC2R(plan, reinterpret_cast<cufftComplex *>(p), p);
        ps.end();
        PM_FFT(ctx, r);
    }
    return PM_OK;
}

int mesh_r2c(pm_ctx *ctx, int f0, int nf) {
    return fft_fields(ctx, ctx->r2c, true, ctx->mesh, ctx->mesh_pad * ctx->P.n_batch, f0, nf);
}
int mesh_c2r(pm_ctx *ctx, int f0, int nf) {
    return fft_fields(ctx, ctx->c2r, false, ctx->mesh, ctx->mesh_pad * ctx->P.n_batch, f0, nf);
}
int lat_r2c(pm_ctx *ctx, int f0, int nf) {
    return fft_fields(ctx, ctx->lr2c, true, ctx->lat, ctx->lat_pad * ctx->P.n_batch, f0, nf);
}
int lat_c2r(pm_ctx *ctx, int f0, int nf) {
    return fft_fields(ctx, ctx->lc2r, false, ctx->lat, ctx->lat_pad * ctx->P.n_batch, f0, nf);
}

PaintArgs paint_args(pm_ctx *ctx, const float *s, const float *mu = nullptr) {
    PaintArgs a{};
    a.g = ctx->g;
    a.s = s;
    a.mu = mu;
    a.mesh = mesh_ref(ctx);
    a.threads = ctx->tune[0];
    return a;
}

bool binned_deposit(const pm_ctx *ctx) { return ctx->dep_ok && ctx->dep_idx && ctx->tune[9] == 2; }

// The binned deposit's buffers, on its first selection (not inside a capture).
int deposit_buffers(pm_ctx *ctx) {
    if (!ctx->dep_ok || ctx->dep_idx) return PM_OK;
    const size_t parts = (size_t)ctx->g.npart * ctx->P.n_batch, bins = (size_t)deposit_tiles(ctx->g) * ctx->P.n_batch;
    if (cudaMalloc(&ctx->dep_key, sizeof(int) * parts) != cudaSuccess ||
        cudaMalloc(&ctx->dep_rank, sizeof(int) * parts) != cudaSuccess ||
        cudaMalloc(&ctx->dep_count, sizeof(int) * bins) != cudaSuccess ||
        cudaMalloc(&ctx->dep_offset, sizeof(int) * (bins + 1)) != cudaSuccess ||
        cudaMalloc(&ctx->dep_chunk, sizeof(int) * deposit_scan_chunks(ctx->g)) != cudaSuccess ||
        cudaMalloc(&ctx->dep_halo, sizeof(float) * deposit_halo_floats(ctx->g)) != cudaSuccess ||
        cudaMemset(ctx->dep_count, 0, sizeof(int) * bins) != cudaSuccess || deposit_prepare() != cudaSuccess ||
        cudaMalloc(&ctx->dep_idx, sizeof(int) * parts) != cudaSuccess) {  // dep_idx last: it marks completion
        cudaGetLastError();
        for (int **p : {&ctx->dep_key, &ctx->dep_rank, &ctx->dep_count, &ctx->dep_offset, &ctx->dep_chunk, &ctx->dep_idx}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        if (ctx->dep_halo) cudaFree(ctx->dep_halo);
        ctx->dep_halo = nullptr;
        return fail(ctx, PM_ENOMEM, "cannot allocate the binned-deposit buffers");
    }
    return PM_OK;
}

// Paint into a plain mesh that this call fills completely, every cell
// starting from `base`: the binned tile-owned deposit (no zeroing), or
// filling and the atomic scatter.
int paint_own(pm_ctx *ctx, int mode, const PaintArgs &pa, float base = 0.f) {
    const bool adj = mode == PAINT_ADJ;
    const int nf = adj ? 4 : 1;
    if (binned_deposit(ctx) && pa.mesh.zs == ctx->P.n_m && pa.mesh.il == (adj ? 4 : 0)) {
        DepositArgs da{};
        da.g = ctx->g;
        da.s = pa.s;
        da.mu = pa.mu;
        da.key = ctx->dep_key;
        da.rank = ctx->dep_rank;
        da.idx = ctx->dep_idx;
        da.count = ctx->dep_count;
        da.offset = ctx->dep_offset;
        da.chunk_sum = ctx->dep_chunk;
        da.mesh = pa.mesh.ptr;
        da.halo = ctx->dep_halo;
        da.tiles = deposit_tiles(ctx->g);
        da.base = base;
        PM_LAUNCH(ctx, "bin_count", launch_bin_count(da, ctx->stream));
        PM_LAUNCH(ctx, "bin_scan_sums", launch_bin_scan_sums(da, ctx->stream));
        PM_LAUNCH(ctx, "bin_scan", launch_bin_scan(da, ctx->stream));
        PM_LAUNCH(ctx, "bin_scatter", launch_bin_scatter(da, ctx->stream));
        PM_LAUNCH(ctx, (adj ? "deposit_adj" : "deposit_density"), launch_deposit(nf, da, ctx->stream));
        PM_LAUNCH(ctx, (adj ? "deposit_halo_4" : "deposit_halo_1"), launch_deposit_halo(nf, da, ctx->stream));
        if (pa.mesh.ptr == ctx->r1) ctx->r1_zero = false;
        if (pa.mesh.ptr == ctx->r4) ctx->r4_zero = false;
        return PM_OK;
    }
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    const bool zeroed = base == 0.f && ((pa.mesh.ptr == ctx->r1 && ctx->r1_zero) || (pa.mesh.ptr == ctx->r4 && ctx->r4_zero));
    if (zeroed)
        ;  // cleared by the previous step's read
    else if (base == 0.f)
        PM_MEMSET(ctx, cudaMemsetAsync(pa.mesh.ptr, 0, sizeof(float) * n3 * nf * ctx->P.n_batch, ctx->stream));
    else
        PM_LAUNCH(ctx, "fill", launch_fill(pa.mesh.ptr, n3 * nf * ctx->P.n_batch, base, ctx->stream));
    if (pa.mesh.ptr == ctx->r1) ctx->r1_zero = false;
    if (pa.mesh.ptr == ctx->r4) ctx->r4_zero = false;
    PM_LAUNCH(ctx, paint_kind(mode), launch_paint(mode, pa, ctx->stream));
    return PM_OK;
}

// The density of s (alpha sum W) into the real scratch field dref.
int paint_density(pm_ctx *ctx, const float *s, const MeshRef &dref) {
    PaintArgs pa = paint_args(ctx, s);
    pa.mesh = dref;
    if (ctx->own) return paint_own(ctx, PAINT_DENSITY, pa);
    PM_MEMSET(ctx, cudaMemsetAsync(dref.ptr, 0, sizeof(float) * density_floats(ctx), ctx->stream));
    PM_LAUNCH(ctx, paint_kind(PAINT_DENSITY), launch_paint(PAINT_DENSITY, pa, ctx->stream));
    return PM_OK;
}

ReadArgs read_args(pm_ctx *ctx, float *s) {
    ReadArgs a{};
    a.g = ctx->g;
    a.s = s;
    a.mesh = mesh_ref(ctx);
    a.table = ctx->d_table;
    a.red_bstride = 2 * (ctx->P.n_steps + 1);
    a.drift_step = -1;
    a.threads = ctx->tune[1];
    return a;
}

// Read arguments after a force evaluation (force_meshes): with the
// potential read, the potential (and psi) meshes instead of the force mesh.
ReadArgs force_read_args(pm_ctx *ctx, float *s) {
    ReadArgs a = read_args(ctx, s);
    if (pot_read(ctx)) {
        a.pot = ctx->rpot;
        int lgn = 0;
        while ((1 << lgn) < ctx->P.n_m) ++lgn;
        a.lgn = lgn;
        a.inv12h = xround_args(ctx).inv12h;
    }
    return a;
}

PreArgs pre_args(pm_ctx *ctx, float *s, float *p) {
    PreArgs a{};
    a.g = ctx->g;
    a.s = s;
    a.p = p;
    a.table = ctx->d_table;
    a.red_bstride = 2 * (ctx->P.n_steps + 1);
    return a;
}

const char *own_kind(int pass, int nf) {
    static const char *names[6][5] = {
        {"", "fft_z_fwd_1", "fft_z_fwd_2", "", "fft_z_fwd_4"}, {"", "fft_y_fwd_1", "fft_y_fwd_2", "", "fft_y_fwd_4"},
        {"", "fft_x_fwd_1", "", "", "fft_x_fwd_4"}, {"", "fft_x_inv_1", "", "fft_x_inv_3", "fft_x_inv_4"},
        {"", "fft_y_inv_1", "fft_y_inv_2", "fft_y_inv_3", "fft_y_inv_4"},
        {"", "fft_z_inv_1", "fft_z_inv_2", "fft_z_inv_3", "fft_z_inv_4"}};
    return names[pass][nf];
}

// Own forward 3D transform of g interleaved real fields into spectrum fields 0 .. g-1.
int own_forward(pm_ctx *ctx, const float *real, int g) {
    PM_LAUNCH(ctx, own_kind(0, g), launch_fft_z_fwd(g, real, ctx->spec, ctx->fg, ctx->stream));
    PM_LAUNCH(ctx, own_kind(1, g), launch_fft_pencils(1, false, ctx->spec, 0, g, ctx->fg, ctx->stream));
    PM_LAUNCH(ctx, own_kind(2, g), launch_fft_pencils(0, false, ctx->spec, 0, g, ctx->fg, ctx->stream));
    return PM_OK;
}

// Own inverse 3D transform of spectrum fields 0 .. g-1 (g = 3, 4: into the
// interleaved r4 layout; g = 1: plain real field).
int own_inverse(pm_ctx *ctx, float *real, int g) {
    PM_LAUNCH(ctx, own_kind(3, g), launch_fft_pencils(0, true, ctx->spec, 0, g, ctx->fg, ctx->stream));
    PM_LAUNCH(ctx, own_kind(4, g), launch_fft_pencils(1, true, ctx->spec, 0, g, ctx->fg, ctx->stream));
    PM_LAUNCH(ctx, own_kind(5, g), launch_fft_z_inv(g, ctx->spec, real, ctx->fg, ctx->stream));
    return PM_OK;
}

// Zero, paint, forward transform(s), spectral
// multiply and inverse transforms; leaves F_x, F_y, F_z (and psi for the
// adjoint) in the scratch fields.  mu != NULL selects the 4-field adjoint
// paint.
int apply_correction(pm_ctx *ctx, double a);
int correction_adjoint(pm_ctx *ctx, double a, int kick_step, int kick_sel);
int64_t nn_cells(pm_ctx *ctx);

int force_meshes(pm_ctx *ctx, const float *s, const float *mu, double a = -1.0, int kick_step = -1, int kick_sel = 0) {
    const bool adj = mu != nullptr;
    const int nf = adj ? 4 : 1;
    const int mode = adj ? PAINT_ADJ : PAINT_DENSITY;
    PaintArgs pa = paint_args(ctx, s, mu);
    if (ctx->own) {
        const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
        float *real = adj ? ctx->r4 : ctx->r1;
        pa.mesh = adj ? mesh_ref(ctx) : density_ref(ctx);
        PM_TRY(paint_own(ctx, mode, pa));
        const int go = adj ? 4 : 3;
        if (pot_pipeline(ctx)) {
            // z and y forward; x round trip to phi (and psi); y and z inverse of
            // those one or two fields; F = S phi on the real mesh into r4.  The
            // adjoint first forms its source v = sum_j S_j u_j on the real mesh
            // (rho, v into rpot) and transforms two fields instead of four,
            // except with the learned correction, whose adjoint reads the
            // painted fields between the transforms
            const int np = adj ? 2 : 1;
            const int nt = adj && !ctx->nn_on ? 2 : nf;
            const float *zin = real;
            if (nt == 2) {
                PM_LAUNCH(ctx, "vjp_source",
                          launch_vjp_source(reinterpret_cast<const float4 *>(ctx->r4), reinterpret_cast<float2 *>(ctx->rpot),
                                            ctx->P.n_m, ctx->P.n_batch, xround_args(ctx).inv12h, ctx->stream));
                zin = ctx->rpot;
            }
            PM_LAUNCH(ctx, own_kind(0, nt), launch_fft_z_fwd(nt, zin, ctx->spec, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, own_kind(1, nt), launch_fft_pencils(1, false, ctx->spec, 0, nt, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, (nt == 4 ? "fft_x_pot_4" : (nt == 2 ? "fft_x_pot_2" : "fft_x_pot_1")),
                      launch_fft_xpot(nt, ctx->spec, ctx->fg, xround_args(ctx), ctx->stream));
            // the correction's adjoint reads the painted (rho, mu) still in r4
            if (adj && ctx->nn_on && a > 0.0) PM_TRY(correction_adjoint(ctx, a, kick_step, kick_sel));
            PM_LAUNCH(ctx, own_kind(4, np), launch_fft_pencils(1, true, ctx->spec, 0, np, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, own_kind(5, np), launch_fft_z_inv(np, ctx->spec, ctx->rpot, ctx->fg, ctx->stream));
            if (!pot_read(ctx))
                PM_LAUNCH(ctx, (adj ? "grad_stencil_2" : "grad_stencil_1"),
                          launch_grad_stencil(ctx->rpot, np, reinterpret_cast<float4 *>(ctx->r4), ctx->P.n_m,
                                              ctx->P.n_batch, xround_args(ctx).inv12h, ctx->stream));
        } else if (x_fused(ctx, adj)) {  // z and y forward, fused x round trip, y and z inverse
            PM_LAUNCH(ctx, own_kind(0, nf), launch_fft_z_fwd(nf, real, ctx->spec, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, own_kind(1, nf), launch_fft_pencils(1, false, ctx->spec, 0, nf, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, (adj ? "fft_x_round_4" : "fft_x_round_1"),
                      launch_fft_xround(adj, ctx->spec, ctx->fg, xround_args(ctx), ctx->stream));
            if (adj && ctx->nn_on && a > 0.0) PM_TRY(correction_adjoint(ctx, a, kick_step, kick_sel));
            PM_LAUNCH(ctx, own_kind(4, go), launch_fft_pencils(1, true, ctx->spec, 0, go, ctx->fg, ctx->stream));
            PM_LAUNCH(ctx, own_kind(5, go), launch_fft_z_inv(go, ctx->spec, ctx->r4, ctx->fg, ctx->stream));
        } else {
            PM_TRY(own_forward(ctx, real, nf));
            PM_LAUNCH(ctx, (adj ? "spectral_adj" : "spectral_force"),
                      launch_spectral(adj ? SPEC_ADJ : SPEC_FORCE, mesh_spec(ctx), ctx->d_pref, ctx->stream));
            // the correction's adjoint reads the painted (rho, mu) still in r4
            if (adj && ctx->nn_on && a > 0.0) PM_TRY(correction_adjoint(ctx, a, kick_step, kick_sel));
            PM_TRY(own_inverse(ctx, ctx->r4, go));
        }
        if (!adj && ctx->nn_on && a > 0.0) PM_TRY(apply_correction(ctx, a));
        if (adj && ctx->nn_on && a > 0.0) {
            const int64_t n4 = nn_cells(ctx);
            PM_LAUNCH(ctx, "nn_add4", launch_add4(reinterpret_cast<float4 *>(ctx->r4),
                                                  reinterpret_cast<const float4 *>(ctx->nn_mesh4), n4, ctx->stream));
        }
        return PM_OK;
    }
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->mesh, 0, sizeof(float) * ctx->mesh_pad * ctx->P.n_batch * nf, ctx->stream));
    PM_LAUNCH(ctx, paint_kind(mode), launch_paint(mode, pa, ctx->stream));
    PM_TRY(mesh_r2c(ctx, 0, nf));
    PM_LAUNCH(ctx, (adj ? "spectral_adj" : "spectral_force"), launch_spectral(adj ? SPEC_ADJ : SPEC_FORCE, mesh_spec(ctx), ctx->d_pref, ctx->stream));
    PM_TRY(mesh_c2r(ctx, 0, adj ? 4 : 3));
    return PM_OK;
}

// The next paint's mesh the read may clear (own transform, potential read:
// the read does not touch r1 or r4; atomic paints, which add into zeros).
float4 *zero_target(pm_ctx *ctx, bool adj, int64_t *n4) {
    if (!ctx->own || !pot_read(ctx) || binned_deposit(ctx)) return nullptr;
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    *n4 = adj ? n3 : n3 / 4;
    return reinterpret_cast<float4 *>(adj ? ctx->r4 : ctx->r1);
}

// Interpolate from the force meshes (particles in lattice order).
int read_forces(pm_ctx *ctx, int mode, const ReadArgs &ra) {
    PM_LAUNCH(ctx, read_kind(mode), launch_read(mode, ra, ctx->stream));
    return PM_OK;
}

// Run `body` (a fixed sequence of launches on the context stream) through a
// cached CUDA graph: the first call with a given key captures it on a
// private stream, later calls replay it on the context stream.  Profiling
// bypasses the graphs (its events are recorded per launch).
int run_graphed(pm_ctx *ctx, int kind, int b, int e, const void *q0, const void *q1, const void *q2, const void *q3,
                const void *q4, uint32_t flags, const std::function<int()> &body) {
    if (!ctx->graphs_on || ctx->prof) return body();
    const void *q[5] = {q0, q1, q2, q3, q4};
    for (auto &g : ctx->graphs) {
        if (g.kind == kind && g.b == b && g.e == e && g.flags == flags && std::equal(q, q + 5, g.q)) {
            PM_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
            ctx->launches += g.launches;
            return PM_OK;
        }
    }
    if (!ctx->cap_stream) PM_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = ctx->stream;
    PM_TRY(pm_set_stream(ctx, ctx->cap_stream));
    cudaError_t ce = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) {
        pm_set_stream(ctx, user);
        return fail(ctx, PM_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(ce));
    }
    const int64_t l0 = ctx->launches;
    const int rc = body();
    cudaGraph_t graph = nullptr;
    ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    pm_set_stream(ctx, user);
    if (rc != PM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return fail(ctx, PM_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ctx, PM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    if (ctx->graphs.size() >= 8) {
        cudaGraphExecDestroy(ctx->graphs.front().exec);
        ctx->graphs.erase(ctx->graphs.begin());
    }
    pm_ctx::GraphEntry ent{kind, b, e, {q0, q1, q2, q3, q4}, flags, exec, ctx->launches - l0};
    ctx->graphs.push_back(ent);
    PM_CUDA(ctx, cudaGraphLaunch(exec, user));
    return PM_OK;
}

double a_of(pm_ctx *ctx, int n) { return step_a(ctx->P, n); }

// Checkpoint slot of step n (steps every, 2 every, ... below n_steps), or -1.
int ck_slot(const pm_ctx *ctx, int n) {
    if (ctx->ck_every <= 0 || n <= 0 || n % ctx->ck_every) return -1;
    return n / ctx->ck_every - 1;
}

int64_t ck_slots(const pm_ctx *ctx, int every) { return every > 0 ? (ctx->P.n_steps - 1) / every : 0; }

// One particle array of all runs: n_batch * n_p^3 * 3 floats.
int64_t state_floats(const pm_ctx *ctx) { return ctx->g.npart * ctx->P.n_batch * 3; }

// which = 0: s_m, 1: p_{m+1/2}.
float *ck_ptr(pm_ctx *ctx, int slot, int which) {
    return ctx->ck_buf + ((int64_t)slot * 2 + which) * state_floats(ctx);
}

int ck_copy(pm_ctx *ctx, float *dst, const float *src) {
    PM_CUDA(ctx, cudaMemcpyAsync(dst, src, sizeof(float) * state_floats(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
    return PM_OK;
}

// Report (and clear) a device-side error flag (a TMA wait that timed out);
// call after a stream synchronisation.
int device_check(pm_ctx *ctx) {
    if (!ctx->d_err) return PM_OK;
    int flag = 0;
    PM_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        PM_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        return fail(ctx, PM_ECUDA, "a bounded device wait (TMA copy of the spectrum) timed out");
    }
    return PM_OK;
}

int check_ptr(pm_ctx *ctx, const void *p, const char *name) {
    if (!p) return fail(ctx, PM_EINVAL, std::string(name) + " must not be NULL");
    if ((uintptr_t)p % 4) return fail(ctx, PM_EINVAL, std::string(name) + " must be 4-byte aligned");
    return PM_OK;
}

int ensure_lattice(pm_ctx *ctx) {
    if (ctx->lat) return PM_OK;
    const size_t bytes = sizeof(float) * (size_t)ctx->lat_pad * ctx->P.n_batch * kLatFields;
    if (cudaMalloc(&ctx->lat, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->lat = nullptr;
        return fail(ctx, PM_ENOMEM, "cannot allocate the initial-condition lattice fields");
    }
    return PM_OK;
}

// White noise -> s1 (fields 0..2), phi (3..8), S (9), s2 (10..12).
int lpt_forward_fields(pm_ctx *ctx, const float *noise, uint64_t seed) {
    PM_TRY(ensure_lattice(ctx));
    const int np = ctx->P.n_p, B = ctx->P.n_batch;
    MeshRef lr = lat_ref(ctx);
    PM_LAUNCH(ctx, "noise", launch_noise(noise, seed, lr, np, B, ctx->stream));
    PM_TRY(lat_r2c(ctx, 0, 1));
    PM_LAUNCH(ctx, "lpt_linear", launch_lpt_linear(lat_spec(ctx), ctx->d_lin, ctx->stream));
    PM_TRY(lat_c2r(ctx, 0, 9));
    PM_LAUNCH(ctx, "lpt_source", launch_lpt_source(lr, np, B, 3, 9, ctx->stream));
    PM_TRY(lat_r2c(ctx, 9, 1));
    PM_LAUNCH(ctx, "lpt_second", launch_lpt_second(lat_spec(ctx), 9, 10, -1.f, ctx->stream));
    PM_TRY(lat_c2r(ctx, 10, 3));
    return PM_OK;
}

// ---------------------------------------------------- learned correction --

int64_t nn_cells(pm_ctx *ctx) { return (int64_t)ctx->P.n_batch * ctx->P.n_m * ctx->P.n_m * ctx->P.n_m; }

int ensure_nn(pm_ctx *ctx) {
    if (ctx->nn_theta) return PM_OK;
    if (!ctx->own) return fail(ctx, PM_ESTATE, "the learned correction needs a power-of-two mesh (own FFT path)");
    const int np = nn_param_count();
    const int64_t cells = nn_cells(ctx);
    const int64_t parts = ctx->g.npart * ctx->P.n_batch;
    const size_t act = (size_t)cells * (NN_IN + 4 * NN_HID + 8);
    if (cudaMalloc(&ctx->nn_theta, sizeof(float) * np) != cudaSuccess ||
        cudaMalloc(&ctx->nn_grad, sizeof(float) * np) != cudaSuccess ||
        cudaMalloc(&ctx->nn_m, sizeof(float) * np) != cudaSuccess ||
        cudaMalloc(&ctx->nn_v, sizeof(float) * np) != cudaSuccess ||
        cudaMalloc(&ctx->nn_packed, nn_packed_bytes()) != cudaSuccess ||
        cudaMalloc(&ctx->nn_act, sizeof(__nv_bfloat16) * act) != cudaSuccess ||
        cudaMalloc(&ctx->nn_part, sizeof(float) * 3 * parts) != cudaSuccess ||
        cudaMalloc(&ctx->nn_loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->nn_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->nn_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->nn_feat, sizeof(__nv_bfloat16) * cells) != cudaSuccess ||
        cudaMalloc(&ctx->nn_mesh4, sizeof(float) * 4 * cells) != cudaSuccess ||
        cudaMalloc(&ctx->nn_gx, sizeof(float) * NN_IN * cells) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PM_ENOMEM, "cannot allocate the learned-correction buffers");
    }
    ctx->nnw = nn_carve(ctx->nn_packed);
    PM_CUDA(ctx, nn_tc_prepare());
    return PM_OK;
}

NNArgs nn_args(pm_ctx *ctx, double a) {
    NNArgs na{};
    na.w = NNWeights{ctx->nnw.w1c, ctx->nnw.w2c, ctx->nnw.w3c, ctx->nnw.w1b,
                     ctx->nnw.w2b, ctx->nnw.w3b, ctx->nnw.b1,  ctx->nnw.b2, ctx->nnw.b3};
    na.err = ctx->nn_err;
    na.feat = ctx->nn_feat;
    na.n = ctx->P.n_m;
    na.rho = ctx->r1;
    na.afeat = (float)a;
    na.pref = ctx->d_pref;
    na.s_scale = (float)((double)ctx->P.n_m * ctx->P.n_m * ctx->P.box);
    na.out = ctx->r4;
    const int64_t cells = nn_cells(ctx);
    na.xg = ctx->nn_act;
    na.h1g = na.xg + cells * NN_IN;
    na.h2g = na.h1g + cells * NN_HID;
    na.g1g = na.h2g + cells * NN_HID;
    na.g2g = na.g1g + cells * NN_HID;
    na.g3g = na.g2g + cells * NN_HID;
    na.grad = ctx->nn_grad;
    na.gb1 = ctx->nn_grad + NN_IN * NN_HID;
    na.gb2 = na.gb1 + NN_HID + NN_HID * NN_HID;
    na.gb3 = na.gb2 + NN_HID + NN_HID * NN_OUT;
    return na;
}

// Report (and clear) a time-out of the tensor-core kernel's MMA waits.
int nn_check(pm_ctx *ctx) {
    int flag = 0;
    PM_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->nn_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) {
        PM_CUDA(ctx, cudaMemset(ctx->nn_err, 0, sizeof(int)));
        return fail(ctx, PM_ECUDA, "tensor-core MMA wait timed out in the learned correction");
    }
    return PM_OK;
}

// Add the network's correction to the force meshes (r4) from the density in
// r1 at scale factor a.
int apply_correction(pm_ctx *ctx, double a) {
    NNArgs na = nn_args(ctx, a);
    na.accumulate = 1;
    PM_LAUNCH(ctx, "nn_feat", launch_nn_feat(ctx->r1, ctx->nn_feat, nn_cells(ctx), ctx->stream));
    PM_LAUNCH(ctx, "nn_fwd_tc", launch_nn_fwd_tc(na, nn_cells(ctx), ctx->stream));
    return PM_OK;
}

// The correction inside an adjoint step, between the forward transforms of
// the 4-field paint (r4 = alpha sum W, sum W mu) and the inverse ones:
// network forward at a (activations kept, dF -> nn_mesh4 slots 0..2),
// backward with the output cotangent s_out c u (c the step's kick factor):
// parameter gradient accumulated, feature cotangents -> density cotangent
// g_rho / c -> nn_mesh4 slot 3; after the inverse transforms nn_mesh4 is
// added to (F, psi), so that the fused read applies the corrected force and
// the full VJP.
int correction_adjoint(pm_ctx *ctx, double a, int kick_step, int kick_sel) {
    const int64_t cells = nn_cells(ctx);
    NNArgs na = nn_args(ctx, a);
    if (!na.w.w1b || !ctx->nn_mesh4 || !ctx->nn_gx || kick_step < 0 || kick_step >= ctx->P.n_steps)
        return fail(ctx, PM_ESTATE, "learned-correction adjoint buffers are not set up");
    na.rho = ctx->r4;
    na.rho_stride = 4;
    na.out = ctx->nn_mesh4;
    na.accumulate = 0;
    PM_LAUNCH(ctx, "nn_feat", launch_nn_feat(ctx->r4, ctx->nn_feat, cells, ctx->stream, 4));
    PM_LAUNCH(ctx, "nn_fwd_train", launch_nn_fwd_tc(na, cells, ctx->stream, true));
    na.gmesh = ctx->r4;
    na.table = ctx->d_table;
    na.kick_step = kick_step;
    na.kick_sel = kick_sel;
    na.nb = ctx->P.n_batch;
    na.gx = ctx->nn_gx;
    PM_LAUNCH(ctx, "nn_bwd", launch_nn_bwd(na, cells, ctx->stream));
    PM_LAUNCH(ctx, "nn_grad_rho", launch_nn_grad_rho(na, ctx->r4, ctx->nn_mesh4, cells, ctx->stream));
    return PM_OK;
}

// Paint the density of s into r1 and evaluate the network into r4 (slots
// 0..2 overwritten); train = also keep the activations.
int nn_forward_at(pm_ctx *ctx, const float *s, double a, bool train) {
    const MeshRef dref = density_ref(ctx);
    PM_TRY(paint_density(ctx, s, dref));
    NNArgs na = nn_args(ctx, a);
    PM_LAUNCH(ctx, "nn_feat", launch_nn_feat(ctx->r1, ctx->nn_feat, nn_cells(ctx), ctx->stream));
    PM_LAUNCH(ctx, (train ? "nn_fwd_train" : "nn_fwd_tc"), launch_nn_fwd_tc(na, nn_cells(ctx), ctx->stream, train));
    return PM_OK;
}

}  // namespace

// ================================================================ C ABI ===

extern "C" {

const char *pm_last_error(const pm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int64_t pm_launch_count(const pm_ctx *ctx) { return ctx ? ctx->launches : 0; }

const int kTuneCand[PM_TUNE_KINDS][3] = {{128, 256, 512}, {128, 256, 512}, {128, 256, 512}, {128, 256, 512},
                                         {8, 16, 0},      {1, 2, 0},       {1, 2, 0},       {1, 2, 3},
                                         {1, 2, 0},       {1, 2, 0}};

static int set_tuning(pm_ctx *ctx, const int *t) {
    for (int k = 0; k < PM_TUNE_KINDS; ++k)
        if (t[k] <= 0 || (t[k] != kTuneCand[k][0] && t[k] != kTuneCand[k][1] && t[k] != kTuneCand[k][2]))
            return fail(ctx, PM_EINVAL,
                        "block sizes must be 128, 256 or 512, the x-pass width 8 or 16, the z stagings 1 or 2, "
                        "the x round trip 1, 2 or 3, the force pipeline 1 or 2, the deposit 1 or 2");
    if (t[9] == 2) PM_TRY(deposit_buffers(ctx));
    for (int k = 0; k < PM_TUNE_KINDS; ++k) ctx->tune[k] = t[k];
    ctx->fg.zthreads = ctx->tune[3];
    ctx->fg.xwidth = ctx->tune[4];
    ctx->fg.ztma = ctx->tune[5] == 2;
    ctx->fg.zstage = ctx->tune[6] == 2;
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);  // captured with the old shapes
    ctx->graphs.clear();
    return PM_OK;
}

int pm_set_tuning(pm_ctx *ctx, const int *threads) {
    if (!ctx || !threads) return fail(ctx, PM_EINVAL, "ctx and threads must not be NULL");
    return set_tuning(ctx, threads);
}

int pm_get_tuning(pm_ctx *ctx, int *threads) {
    if (!ctx || !threads) return fail(ctx, PM_EINVAL, "ctx and threads must not be NULL");
    for (int k = 0; k < PM_TUNE_KINDS; ++k) threads[k] = ctx->tune[k];
    return PM_OK;
}

int pm_autotune(pm_ctx *ctx, const float *s, float *ms) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    DeviceGuard guard(ctx->device);
    const int B = ctx->P.n_batch;
    const int64_t npart = ctx->g.npart * B;
    float *f = nullptr;
    if (cudaMalloc(&f, sizeof(float) * 3 * npart) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PM_ENOMEM, "cannot allocate the autotuner's scratch force");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = ctx->prof;
    ctx->prof = false;
    int rc = PM_OK;
    // one representative launch sequence per family, on the context's own
    // scratch meshes filled by a real force evaluation of s
    auto body = [&](int kind) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (kind == 0) {
            PaintArgs pa = paint_args(ctx, s);
            pa.mesh = density_ref(ctx);
            if ((e = launch_paint(PAINT_DENSITY, pa, ctx->stream)) != cudaSuccess) return e;
            pa = paint_args(ctx, s, s);
            return launch_paint(PAINT_ADJ, pa, ctx->stream);
        }
        if (kind == 1) {
            ReadArgs ra = force_read_args(ctx, const_cast<float *>(s));
            ra.f = f;
            return launch_read(READ_FORCE, ra, ctx->stream);
        }
        if (kind == 2) {
            if ((e = launch_spectral(SPEC_FORCE, mesh_spec(ctx), ctx->d_pref, ctx->stream)) != cudaSuccess) return e;
            return launch_spectral(SPEC_ADJ, mesh_spec(ctx), ctx->d_pref, ctx->stream);
        }
        if (kind == 4) {
            if ((e = launch_fft_pencils(0, false, ctx->spec, 0, 4, ctx->fg, ctx->stream)) != cudaSuccess) return e;
            return launch_fft_pencils(0, true, ctx->spec, 0, 4, ctx->fg, ctx->stream);
        }
        if (kind == 6) return launch_fft_z_fwd(4, ctx->r4, ctx->spec, ctx->fg, ctx->stream);
        if (kind == 7) {  // the x side of a force and an adjoint evaluation
            for (int adj = 0; adj < 2 && e == cudaSuccess; ++adj) {
                if (x_fused(ctx, adj != 0)) {
                    e = launch_fft_xround(adj != 0, ctx->spec, ctx->fg, xround_args(ctx), ctx->stream);
                    continue;
                }
                if ((e = launch_fft_pencils(0, false, ctx->spec, 0, adj ? 4 : 1, ctx->fg, ctx->stream)) != cudaSuccess)
                    return e;
                if ((e = launch_spectral(adj ? SPEC_ADJ : SPEC_FORCE, mesh_spec(ctx), ctx->d_pref, ctx->stream)) !=
                    cudaSuccess)
                    return e;
                e = launch_fft_pencils(0, true, ctx->spec, 0, adj ? 4 : 3, ctx->fg, ctx->stream);
            }
            return e;
        }
        if (kind == 5) {  // the z inverses the force pipeline runs
            if (pot_pipeline(ctx)) {
                if ((e = launch_fft_z_inv(2, ctx->spec, ctx->rpot, ctx->fg, ctx->stream)) != cudaSuccess) return e;
                return launch_fft_z_inv(1, ctx->spec, ctx->rpot, ctx->fg, ctx->stream);
            }
            if ((e = launch_fft_z_inv(3, ctx->spec, ctx->r4, ctx->fg, ctx->stream)) != cudaSuccess) return e;
            return launch_fft_z_inv(4, ctx->spec, ctx->r4, ctx->fg, ctx->stream);
        }
        if (kind == 9) {  // a density paint and an adjoint paint, each filling its mesh
            PaintArgs pa = paint_args(ctx, s);
            pa.mesh = density_ref(ctx);
            if (paint_own(ctx, PAINT_DENSITY, pa) != PM_OK) return cudaErrorUnknown;
            pa = paint_args(ctx, s, s);
            pa.mesh = mesh_ref(ctx);
            if (paint_own(ctx, PAINT_ADJ, pa) != PM_OK) return cudaErrorUnknown;
            return cudaGetLastError();
        }
        if (kind == 8) {  // a whole force evaluation with its read, and an adjoint one (the pipelines differ
                          // from the x pass on; the potential read moves the difference into the read)
            if (force_meshes(ctx, s, nullptr) != PM_OK) return cudaErrorUnknown;
            ReadArgs ra = force_read_args(ctx, const_cast<float *>(s));
            ra.f = f;
            if ((e = launch_read(READ_FORCE, ra, ctx->stream)) != cudaSuccess) return e;
            if (force_meshes(ctx, s, s) != PM_OK) return cudaErrorUnknown;
            return cudaGetLastError();
        }
        if ((e = launch_fft_z_fwd(1, ctx->r1, ctx->spec, ctx->fg, ctx->stream)) != cudaSuccess) return e;
        if ((e = launch_fft_z_fwd(4, ctx->r4, ctx->spec, ctx->fg, ctx->stream)) != cudaSuccess) return e;
        if ((e = launch_fft_z_inv(3, ctx->spec, ctx->r4, ctx->fg, ctx->stream)) != cudaSuccess) return e;
        return launch_fft_z_inv(4, ctx->spec, ctx->r4, ctx->fg, ctx->stream);
    };
    int best[PM_TUNE_KINDS];
    for (int k = 0; k < PM_TUNE_KINDS; ++k) best[k] = ctx->tune[k];
    rc = force_meshes(ctx, s, nullptr);
    for (int kind = 0; kind < PM_TUNE_KINDS && rc == PM_OK; ++kind) {
        if ((kind == 3 && !(ctx->own && ctx->P.n_m >= 256)) || (kind == 4 && !ctx->own) ||
            (kind == 5 && !(ctx->own && ctx->zmaps[0].valid)) || (kind == 6 && !ctx->own) ||
            (kind == 7 && !ctx->own) ||
            (kind == 8 && !(ctx->own && !(ctx->P.solver & PM_SOLVER_SPECTRAL_GRADIENT))) ||
            (kind == 9 && !ctx->dep_ok)) {
            if (ms) ms[3 * kind] = ms[3 * kind + 1] = ms[3 * kind + 2] = 0.f;
            continue;
        }
        float best_ms = 0.f;
        if (ms) ms[3 * kind + 2] = 0.f;
        for (int c = 0; c < 3 && rc == PM_OK && kTuneCand[kind][c]; ++c) {
            int t[PM_TUNE_KINDS];
            for (int k = 0; k < PM_TUNE_KINDS; ++k) t[k] = best[k];
            t[kind] = kTuneCand[kind][c];
            if ((rc = set_tuning(ctx, t)) != PM_OK) break;
            cudaError_t e = body(kind);  // warm-up (first use of this variant)
            cudaEventRecord(e0, ctx->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = body(kind);
            cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = fail(ctx, PM_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
            float t_ms = 0.f;
            cudaEventElapsedTime(&t_ms, e0, e1);
            t_ms /= 3.f;
            if (ms) ms[3 * kind + c] = t_ms;
            if (c == 0 || t_ms < best_ms) {
                best_ms = t_ms;
                best[kind] = kTuneCand[kind][c];
            }
        }
    }
    if (rc == PM_OK) rc = set_tuning(ctx, best);
    ctx->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(f);
    return rc;
}

int pm_use_graphs(pm_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    ctx->graphs_on = enable != 0;
    return PM_OK;
}

int pm_inject_wait_timeout(pm_ctx *ctx, int which) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    if (which != 0 && which != 1) return fail(ctx, PM_EINVAL, "which must be 0 (spectrum copy) or 1 (correction MMA)");
    int *flag = which == 0 ? ctx->d_err : ctx->nn_err;
    if (!flag)
        return fail(ctx, PM_ESTATE, which == 0 ? "this context has no bounded copy wait (library FFT not in use)"
                                               : "set the network parameters first");
    DeviceGuard guard(ctx->device);
    PM_CUDA(ctx, cudaMemsetAsync(flag, 1, sizeof(int), ctx->stream));  // any non-zero word: timed out
    return PM_OK;
}

int64_t pm_checkpoint_floats(const pm_ctx *ctx, int32_t every) {
    if (!ctx || every < 0) return -1;
    return ck_slots(ctx, every) * 2 * state_floats(ctx);
}

int pm_set_checkpoints(pm_ctx *ctx, int32_t every, float *ckpt) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    if (every < 0) return fail(ctx, PM_EINVAL, "every must be >= 0");
    if (ck_slots(ctx, every) > 0) PM_TRY(check_ptr(ctx, ckpt, "ckpt"));
    ctx->ck_every = ck_slots(ctx, every) > 0 ? every : 0;
    ctx->ck_buf = ctx->ck_every ? ckpt : nullptr;
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);  // captured with the old copies
    ctx->graphs.clear();
    return PM_OK;
}

int pm_profile(pm_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    ctx->prof = enable != 0;
    return PM_OK;
}

int pm_profile_kinds(const pm_ctx *ctx) { return ctx ? (int)ctx->kinds.size() : 0; }

const char *pm_profile_name(const pm_ctx *ctx, int kind) {
    if (!ctx || kind < 0 || kind >= (int)ctx->kinds.size()) return "";
    return ctx->kinds[kind].c_str();
}

int pm_profile_read(pm_ctx *ctx, int64_t *counts, double *ms, int n) {
    if (!ctx || (n > 0 && (!counts || !ms))) return fail(ctx, PM_EINVAL, "bad arguments");
    DeviceGuard guard(ctx->device);
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PM_TRY(device_check(ctx));  // a bounded TMA wait that timed out
    for (int i = 0; i < n; ++i) {
        counts[i] = 0;
        ms[i] = 0.0;
    }
    for (size_t r = 0; r < ctx->rec_kind.size(); ++r) {
        float t = 0.f;
        PM_CUDA(ctx, cudaEventElapsedTime(&t, ctx->pool[2 * r], ctx->pool[2 * r + 1]));
        const int k = ctx->rec_kind[r];
        if (k < n) {
            counts[k] += 1;
            ms[k] += t;
        }
    }
    ctx->rec_kind.clear();
    ctx->pool_used = 0;
    return PM_OK;
}

int pm_create(const pm_config *cfg, pm_ctx **out) {
    if (!out) return fail(nullptr, PM_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, PM_EINVAL, "cfg must not be NULL");
    const pm_config &c = *cfg;
    if (c.n_p < 2 || c.n_p % 2 || c.n_p > 4096) return fail(nullptr, PM_EINVAL, "n_p must be even, 2..4096");
    if (c.n_m < 4 || c.n_m % 2 || c.n_m > 4096) return fail(nullptr, PM_EINVAL, "n_m must be even, 4..4096");
    if (c.n_batch < 1 || c.n_batch > 65535) return fail(nullptr, PM_EINVAL, "n_batch must be 1..65535");
    if (c.n_steps < 1 || c.n_steps > 100000) return fail(nullptr, PM_EINVAL, "n_steps must be 1..100000");
    if (!(c.box > 0)) return fail(nullptr, PM_EINVAL, "box must be > 0");
    if (!(c.a_init > 0 && c.a_final > c.a_init)) return fail(nullptr, PM_EINVAL, "need 0 < a_init < a_final");
    if (!(c.h > 0)) return fail(nullptr, PM_EINVAL, "h must be > 0");
    if (c.solver & ~31) return fail(nullptr, PM_EINVAL, "unknown solver flag");
    {
        int rc = check_cosmology(nullptr, c.omega_m, c.sigma8, c.n_batch, c.solver);
        if (!rc) rc = check_emulator_range(c.a_init, c.a_final, c.solver);
        if (rc) return rc;
    }
    const int64_t npart = (int64_t)c.n_p * c.n_p * c.n_p;
    if (npart * c.n_batch * 3 > ((int64_t)1 << 40)) return fail(nullptr, PM_ERANGE, "too many particles");

    pm_ctx *ctx = new pm_ctx();
    ctx->P = Params{c.n_p, c.n_m, c.n_batch, c.n_steps, c.box, c.a_init, c.a_final, c.h, c.n_s, c.solver};
    ctx->om.assign(c.omega_m, c.omega_m + c.n_batch);
    ctx->s8.assign(c.sigma8, c.sigma8 + c.n_batch);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, PM_ECUDA, "no CUDA device");
    }
    ctx->g.np = c.n_p;
    ctx->g.nm = c.n_m;
    ctx->g.nb = c.n_batch;
    ctx->g.order = (c.solver & PM_SOLVER_TSC) ? 3 : 2;
    ctx->g.npart = npart;
    ctx->g.ratio = (c.n_m % c.n_p == 0) ? c.n_m / c.n_p : 0;
    ctx->g.inv_np = 1.0f / c.n_p;
    ctx->g.inv_h = (float)(c.n_m / c.box);
    ctx->g.alpha = (float)std::pow((double)c.n_m / c.n_p, 3);
    ctx->mesh_pad = padded(c.n_m);
    ctx->lat_pad = padded(c.n_p);

    auto bail = [&](int code) {
        std::string msg = ctx->err;
        pm_destroy(ctx);
        g_create_error = msg;
        return code;
    };
    const int B = c.n_batch;
    ctx->own = own_fft_supported(c.n_m);
    if (ctx->own) {
        const int n = c.n_m;
        ctx->fg.n = n;
        ctx->fg.nb = B;
        ctx->fg.zc = own_fft_zc(n);
        ctx->fg.fstride = (int64_t)B * n * n * ctx->fg.zc;
        const size_t n3 = (size_t)n * n * n;
        if (cudaMalloc(&ctx->r1, sizeof(float) * n3 * B) != cudaSuccess ||
            cudaMalloc(&ctx->r4, sizeof(float) * 4 * n3 * B) != cudaSuccess ||
            cudaMalloc(&ctx->rpot, sizeof(float) * 2 * n3 * B) != cudaSuccess ||
            cudaMalloc(&ctx->spec, sizeof(float2) * 4 * (size_t)ctx->fg.fstride) != cudaSuccess ||
            cudaMalloc(&ctx->tw, sizeof(float2) * 1024) != cudaSuccess ||
            cudaMemset(ctx->spec, 0, sizeof(float2) * 4 * (size_t)ctx->fg.fstride) != cudaSuccess ||
            upload_fft_constants(ctx->tw) != cudaSuccess) {
            cudaGetLastError();
            fail(ctx, PM_ENOMEM, "cannot allocate the FFT meshes");
            return bail(PM_ENOMEM);
        }
        ctx->fg.tw = ctx->tw;
        if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            fail(ctx, PM_ENOMEM, "cannot allocate the device error flag");
            return bail(PM_ENOMEM);
        }
        ctx->fg.err = ctx->d_err;
        ctx->fg.tmaps = ctx->zmaps;
        ctx->fg.ztma = encode_z_inv_maps(ctx->spec, ctx->fg, ctx->zmaps) ? 1 : 0;
        ctx->tune[5] = ctx->fg.ztma ? 2 : 1;
        ctx->tune[7] = ctx->P.n_m >= 512 ? 3 : 2;  // the fused adjoint spills on lines of 512+ points
        // the potential pipeline needs the 4-point difference gradient
        ctx->tune[8] = (c.solver & PM_SOLVER_SPECTRAL_GRADIENT) ? 1 : 2;
        ctx->dep_ok = deposit_supported(ctx->g, n);  // buffers on first selection (tuning family [9])
    } else if (cudaMalloc(&ctx->mesh, sizeof(float) * (size_t)ctx->mesh_pad * B * kMeshFields) != cudaSuccess) {
        cudaGetLastError();
        fail(ctx, PM_ENOMEM, "cannot allocate the FFT meshes");
        return bail(PM_ENOMEM);
    }
    if (cudaMalloc(&ctx->d_table, sizeof(float4) * (size_t)c.n_steps * B) != cudaSuccess ||
        cudaMalloc(&ctx->d_pref, sizeof(float) * B) != cudaSuccess ||
        cudaMalloc(&ctx->d_grad, sizeof(float) * ctx->P.n_m) != cudaSuccess ||
        cudaMalloc(&ctx->d_dec, sizeof(float) * ctx->P.n_m) != cudaSuccess ||
        cudaMalloc(&ctx->d_fac, sizeof(float4) * B) != cudaSuccess ||
        cudaMalloc(&ctx->d_lin, sizeof(LinParams) * B) != cudaSuccess ||
        cudaMalloc(&ctx->d_red, sizeof(double) * B * 2 * (c.n_steps + 1)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pk, sizeof(double) * B * 3 * (c.n_m / 2)) != cudaSuccess ||
        cudaMalloc(&ctx->d_lred, sizeof(double) * B * 8) != cudaSuccess) {
        cudaGetLastError();
        fail(ctx, PM_ENOMEM, "device allocation failed in pm_create");
        return bail(PM_ENOMEM);
    }
    {
        // D(k) = (8 sin(k h) - sin(2 k h)) / (6 h) per axis index, k = 2 pi n_j / L
        // (k itself with the spectral-gradient flag; 0 at the Nyquist index);
        // deconvolution 1 / sinc^4(k h / 2) per axis (1 without the flag)
        std::vector<float> grad(c.n_m), dec(c.n_m);
        const double h = c.box / c.n_m;
        for (int j = 0; j < c.n_m; ++j) {
            const int nj = j < c.n_m / 2 ? j : j - c.n_m;
            const double kh = 2.0 * M_PI * nj / c.n_m;
            const double d = (c.solver & PM_SOLVER_SPECTRAL_GRADIENT) ? kh / h
                                                                       : (8.0 * std::sin(kh) - std::sin(2.0 * kh)) / (6.0 * h);
            grad[j] = 2 * j == c.n_m ? 0.f : (float)d;
            const double x = 0.5 * kh, sc = nj == 0 ? 1.0 : std::sin(x) / x;
            const double win = std::pow(sc, (c.solver & PM_SOLVER_TSC) ? 6.0 : 4.0);  // paint and read windows
            dec[j] = (c.solver & PM_SOLVER_DECONVOLVE) ? (float)(1.0 / win) : 1.f;
        }
        if (cudaMemcpy(ctx->d_grad, grad.data(), sizeof(float) * c.n_m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->d_dec, dec.data(), sizeof(float) * c.n_m, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            fail(ctx, PM_ECUDA, "cannot upload the gradient table");
            return bail(PM_ECUDA);
        }
    }
    int rc = upload_tables(ctx);
    if (rc) return bail(rc);
    size_t ws[4] = {0, 0, 0, 0};
    if ((!ctx->own && (rc = make_plan(ctx, &ctx->r2c, c.n_m, true, B, &ws[0]))) ||
        (!ctx->own && (rc = make_plan(ctx, &ctx->c2r, c.n_m, false, B, &ws[1]))) ||
        (rc = make_plan(ctx, &ctx->lr2c, c.n_p, true, B, &ws[2])) ||
        (rc = make_plan(ctx, &ctx->lc2r, c.n_p, false, B, &ws[3])))
        return bail(rc);
    ctx->have_plans = true;
    size_t wmax = 0;
    for (size_t w : ws) wmax = w > wmax ? w : wmax;
    if (wmax) {
        if (cudaMalloc(&ctx->work, wmax) != cudaSuccess) {
            cudaGetLastError();
            fail(ctx, PM_ENOMEM, "cannot allocate the cuFFT work area");
            return bail(PM_ENOMEM);
        }
    }
    for (cufftHandle h : {ctx->r2c, ctx->c2r, ctx->lr2c, ctx->lc2r}) {
        if (h && cufftSetWorkArea(h, ctx->work) != CUFFT_SUCCESS) {
            fail(ctx, PM_ECUFFT, "cufftSetWorkArea failed");
            return bail(PM_ECUFFT);
        }
    }
    rc = pm_set_stream(ctx, nullptr);
    if (rc) return bail(rc);
    *out = ctx;
    return PM_OK;
}

int pm_destroy(pm_ctx *ctx) {
    if (!ctx) return PM_OK;
    DeviceGuard guard(ctx->device);
    if (ctx->have_plans || ctx->r2c) {
        for (cufftHandle h : {ctx->r2c, ctx->c2r, ctx->lr2c, ctx->lc2r})
            if (h) cufftDestroy(h);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    for (void *p : {(void *)ctx->nn_packed, (void *)ctx->nn_theta, (void *)ctx->nn_grad, (void *)ctx->nn_m,
                    (void *)ctx->nn_v, (void *)ctx->nn_part, (void *)ctx->nn_act, (void *)ctx->nn_loss,
                    (void *)ctx->nn_err, (void *)ctx->nn_feat, (void *)ctx->nn_mesh4, (void *)ctx->nn_gx})
        if (p) cudaFree(p);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (void *p : {(void *)ctx->r1, (void *)ctx->r4, (void *)ctx->rpot, (void *)ctx->spec, (void *)ctx->tw,
                    (void *)ctx->d_err})
        if (p) cudaFree(p);
    for (void *p : {(void *)ctx->dep_key, (void *)ctx->dep_rank, (void *)ctx->dep_idx, (void *)ctx->dep_count,
                    (void *)ctx->dep_offset, (void *)ctx->dep_chunk, (void *)ctx->dep_halo})
        if (p) cudaFree(p);
    for (void *p : {(void *)ctx->mesh, (void *)ctx->lat, (void *)ctx->d_table, (void *)ctx->d_pref, (void *)ctx->d_grad, (void *)ctx->d_dec,
                    (void *)ctx->d_fac, (void *)ctx->d_lin, (void *)ctx->d_red, (void *)ctx->d_pk,
                    (void *)ctx->d_lred, ctx->work})
        if (p) cudaFree(p);
    delete ctx;
    return PM_OK;
}

int pm_set_stream(pm_ctx *ctx, void *stream) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    ctx->stream = static_cast<cudaStream_t>(stream);
    for (cufftHandle h : {ctx->r2c, ctx->c2r, ctx->lr2c, ctx->lc2r})
        if (h) PM_FFT(ctx, cufftSetStream(h, ctx->stream));
    return PM_OK;
}

int pm_set_cosmology(pm_ctx *ctx, const double *omega_m, const double *sigma8) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    DeviceGuard guard(ctx->device);
    PM_TRY(check_cosmology(ctx, omega_m, sigma8, ctx->P.n_batch, ctx->P.solver));
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->om.assign(omega_m, omega_m + ctx->P.n_batch);
    ctx->s8.assign(sigma8, sigma8 + ctx->P.n_batch);
    return upload_tables(ctx);
}

int pm_get_coefficients(pm_ctx *ctx, double *out, double *dout) {
    if (!ctx || !out) return fail(ctx, PM_EINVAL, "ctx and out must not be NULL");
    const int N = ctx->P.n_steps;
    for (int b = 0; b < ctx->P.n_batch; ++b)
        for (int n = 0; n < N; ++n) {
            const HostTables &t = ctx->tabs[b];
            double *o = out + ((size_t)b * N + n) * 3;
            o[0] = t.ka[n];
            o[1] = t.dr[n];
            o[2] = t.kb[n];
            if (dout) {
                double *d = dout + ((size_t)b * N + n) * 3;
                d[0] = t.dka[n];
                d[1] = t.ddr[n];
                d[2] = t.dkb[n];
            }
        }
    return PM_OK;
}

int pm_host_coefficients(const pm_config *cfg, double *kdk, double *dkdk, double *lpt, double *amp) {
    if (!cfg) return fail(nullptr, PM_EINVAL, "cfg must not be NULL");
    if (cfg->n_batch < 1 || cfg->n_steps < 1 || !(cfg->a_init > 0 && cfg->a_final > cfg->a_init))
        return fail(nullptr, PM_EINVAL, "bad n_batch, n_steps or a range");
    if (cfg->solver & ~31) return fail(nullptr, PM_EINVAL, "unknown solver flag");
    {
        int rc = check_cosmology(nullptr, cfg->omega_m, cfg->sigma8, cfg->n_batch, cfg->solver);
        if (!rc) rc = check_emulator_range(cfg->a_init, cfg->a_final, cfg->solver);
        if (rc) return rc;
    }
    Params P{cfg->n_p, cfg->n_m, cfg->n_batch, cfg->n_steps, cfg->box, cfg->a_init, cfg->a_final, cfg->h, cfg->n_s,
             cfg->solver};
    const int N = cfg->n_steps;
    for (int b = 0; b < cfg->n_batch; ++b) {
        HostTables t;
        host_tables(P, cfg->omega_m[b], cfg->sigma8[b], &t);
        for (int n = 0; n < N; ++n) {
            const size_t o = ((size_t)b * N + n) * 3;
            if (kdk) {
                kdk[o] = t.ka[n];
                kdk[o + 1] = t.dr[n];
                kdk[o + 2] = t.kb[n];
            }
            if (dkdk) {
                dkdk[o] = t.dka[n];
                dkdk[o + 1] = t.ddr[n];
                dkdk[o + 2] = t.dkb[n];
            }
        }
        if (lpt)
            for (int i = 0; i < 4; ++i) lpt[4 * b + i] = t.lpt[i];
        if (amp) {
            amp[2 * b] = t.amp;
            amp[2 * b + 1] = t.dlnamp;
        }
    }
    return PM_OK;
}

int pm_force(pm_ctx *ctx, const float *s, float *f) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, f, "f"));
    DeviceGuard guard(ctx->device);
    PM_TRY(force_meshes(ctx, s, nullptr));
    ReadArgs ra = force_read_args(ctx, const_cast<float *>(s));
    ra.f = f;
    return read_forces(ctx, READ_FORCE, ra);
}

int pm_kdk_step(pm_ctx *ctx, int32_t step, float *s, float *p, float *f) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, p, "p"));
    PM_TRY(check_ptr(ctx, f, "f"));
    if (step < 0 || step >= ctx->P.n_steps) return fail(ctx, PM_EINVAL, "step out of range");
    DeviceGuard guard(ctx->device);
    PreArgs pr = pre_args(ctx, s, p);
    pr.f = f;
    pr.step = step;
    PM_LAUNCH(ctx, "pre_kick_drift", launch_pre(PRE_KICK_DRIFT, pr, ctx->stream));
    PM_TRY(force_meshes(ctx, s, nullptr, a_of(ctx, step + 1)));
    ReadArgs ra = force_read_args(ctx, s);
    ra.p = p;
    ra.f = f;
    ra.kick_step = step;
    ra.kick_sel = KICK_B;
    return read_forces(ctx, READ_HALF_KICK, ra);
}

int pm_integrate(pm_ctx *ctx, int32_t step_begin, int32_t step_end, float *s, float *p, float *f) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, p, "p"));
    PM_TRY(check_ptr(ctx, f, "f"));
    if (step_begin < 0 || step_end > ctx->P.n_steps || step_begin >= step_end)
        return fail(ctx, PM_EINVAL, "need 0 <= step_begin < step_end <= n_steps");
    DeviceGuard guard(ctx->device);
    return run_graphed(ctx, 1, step_begin, step_end, s, p, f, nullptr, nullptr, 0, [&]() -> int {
        ReadArgs ra = force_read_args(ctx, s);
        ra.p = p;
        ra.f = f;
        ctx->r1_zero = false;
        for (int n = step_begin; n < step_end; ++n) {
            PM_TRY(force_meshes(ctx, s, nullptr, a_of(ctx, n)));
            const int ck = ck_slot(ctx, n);
            if (ck >= 0) PM_TRY(ck_copy(ctx, ck_ptr(ctx, ck, 0), s));  // s_n
            ra.kick_step = n;
            ra.kick_sel = n == step_begin ? KICK_A : KICK_MERGED;
            ra.drift_step = n;
            ra.zero = zero_target(ctx, false, &ra.zero4);  // the density mesh, for the next step's paint
            PM_TRY(read_forces(ctx, READ_KICK_DRIFT, ra));
            ctx->r1_zero = ra.zero != nullptr;
            if (ck >= 0) PM_TRY(ck_copy(ctx, ck_ptr(ctx, ck, 1), p));  // p_{n+1/2}
        }
        PM_TRY(force_meshes(ctx, s, nullptr, a_of(ctx, step_end)));
        ra.kick_step = step_end - 1;
        ra.kick_sel = KICK_B;
        ra.drift_step = -1;
        ra.zero = nullptr;
        ctx->r1_zero = false;
        return read_forces(ctx, READ_HALF_KICK, ra);
    });
}

// Reverse time: the state enters at a[step_end].  Each iteration n paints at
// s_n, whose reverse drift was applied by the previous read (or by the
// opening pre-kernel), and its read both finishes step n (VJP, undo of the
// merged kick) and applies the reverse drift of step n - 1.
int pm_adjoint_integrate(pm_ctx *ctx, int32_t step_begin, int32_t step_end, float *s, float *p, const float *f,
                         float *lam, float *mu, double *domega, uint32_t flags) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, p, "p"));
    PM_TRY(check_ptr(ctx, f, "f"));
    PM_TRY(check_ptr(ctx, lam, "lam"));
    PM_TRY(check_ptr(ctx, mu, "mu"));
    if (step_begin < 0 || step_end > ctx->P.n_steps || step_begin >= step_end)
        return fail(ctx, PM_EINVAL, "need 0 <= step_begin < step_end <= n_steps");
    DeviceGuard guard(ctx->device);
    const int N = ctx->P.n_steps, B = ctx->P.n_batch;
    const int last = step_end - 1;
    PM_TRY(run_graphed(ctx, 2, step_begin, step_end, s, p, f, lam, mu, flags, [&]() -> int {
        ctx->r4_zero = false;
        PM_MEMSET(ctx, cudaMemsetAsync(ctx->d_red, 0, sizeof(double) * B * 2 * (N + 1), ctx->stream));
        if (ctx->nn_on)  // parameter gradient of this adjoint run
            PM_MEMSET(ctx, cudaMemsetAsync(ctx->nn_grad, 0, sizeof(float) * nn_param_count(), ctx->stream));
        if (flags & PM_ADJ_MU_ZERO) {
            // undo the last half kick with the stored F(s_N) (mu = 0: no VJP)
            PM_LAUNCH(ctx, "kick", launch_kick(ctx->g, p, f, ctx->d_table, last, KICK_B, -1.f, ctx->stream));
            PreArgs pr = pre_args(ctx, s, p);
            pr.lam = lam;
            pr.mu = mu;
            pr.step = last;
            pr.red = ctx->d_red + 2 * last + 1;
            PM_LAUNCH(ctx, "pre_rev_drift", launch_pre(PRE_REV_DRIFT, pr, ctx->stream));
        } else {
            // VJP of the last half kick at s_N, fused with the reverse drift of step `last`
            PM_TRY(force_meshes(ctx, s, mu, a_of(ctx, last + 1), last, KICK_B));
            ReadArgs ra = force_read_args(ctx, s);
            ra.p = p;
            ra.lam = lam;
            ra.mu = mu;
            ra.kick_step = last;
            ra.kick_sel = KICK_B;
            ra.drift_step = last;
            ra.red = ctx->d_red + 2 * N;
            ra.red2_offset = (2 * last + 1) - 2 * N;
            ra.zero = zero_target(ctx, true, &ra.zero4);  // the 4-field mesh, for the next step's paint
            PM_TRY(read_forces(ctx, READ_ADJ, ra));
            ctx->r4_zero = ra.zero != nullptr;
        }
        for (int n = last; n >= step_begin; --n) {
            const int ck = ck_slot(ctx, n);
            if (ck >= 0) {  // the loop holds (s_n, p_{n+1/2}) here: take the forward run's copies
                PM_TRY(ck_copy(ctx, s, ck_ptr(ctx, ck, 0)));
                PM_TRY(ck_copy(ctx, p, ck_ptr(ctx, ck, 1)));
            }
            PM_TRY(force_meshes(ctx, s, mu, a_of(ctx, n), n, n == step_begin ? KICK_A : KICK_MERGED));
            ReadArgs ra = force_read_args(ctx, s);
            ra.p = p;
            ra.lam = lam;
            ra.mu = mu;
            ra.kick_step = n;
            ra.kick_sel = n == step_begin ? KICK_A : KICK_MERGED;
            ra.red = ctx->d_red + 2 * n;
            if (n > step_begin) {
                ra.drift_step = n - 1;
                ra.red2_offset = (2 * (n - 1) + 1) - 2 * n;
            }
            ra.zero = n > step_begin ? zero_target(ctx, true, &ra.zero4) : nullptr;
            PM_TRY(read_forces(ctx, READ_ADJ, ra));
            ctx->r4_zero = ra.zero != nullptr;
        }
        ctx->r4_zero = false;
        return PM_OK;
    }));
    if (domega) {
        std::vector<double> red((size_t)B * 2 * (N + 1));
        PM_CUDA(ctx, cudaMemcpyAsync(red.data(), ctx->d_red, sizeof(double) * red.size(), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        PM_TRY(device_check(ctx));
        for (int b = 0; b < B; ++b) {
            const HostTables &t = ctx->tabs[b];
            const double om = ctx->om[b];
            const double *r = red.data() + (size_t)b * 2 * (N + 1);
            double acc = 0.0;
            for (int n = step_begin; n < step_end; ++n) {
                const double c = t.ka[n] + (n > step_begin ? t.kb[n - 1] : 0.0);
                const double dc = t.dka[n] + (n > step_begin ? t.dkb[n - 1] : 0.0);
                acc += r[2 * n] * (dc + c / om) + r[2 * n + 1] * t.ddr[n];
            }
            acc += r[2 * N] * (t.dkb[last] + t.kb[last] / om);
            domega[b] = acc;
        }
    }
    return PM_OK;
}

int pm_init_lpt(pm_ctx *ctx, const float *noise, uint64_t seed, float *s, float *p) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, p, "p"));
    if (noise) PM_TRY(check_ptr(ctx, noise, "noise"));
    DeviceGuard guard(ctx->device);
    PM_TRY(lpt_forward_fields(ctx, noise, seed));
    PM_LAUNCH(ctx, "lpt_combine", launch_lpt_combine(lat_ref(ctx), ctx->P.n_p, ctx->P.n_batch, ctx->d_fac, s, p, ctx->stream));
    return PM_OK;
}

int pm_init_lpt_adjoint(pm_ctx *ctx, const float *noise, uint64_t seed, const float *lam, const float *mu,
                        float *dnoise, double *dcosmo) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, lam, "lam"));
    PM_TRY(check_ptr(ctx, mu, "mu"));
    if (noise) PM_TRY(check_ptr(ctx, noise, "noise"));
    if (dnoise) PM_TRY(check_ptr(ctx, dnoise, "dnoise"));
    DeviceGuard guard(ctx->device);
    const int np = ctx->P.n_p, B = ctx->P.n_batch;
    PM_TRY(lpt_forward_fields(ctx, noise, seed));
    MeshRef lr = lat_ref(ctx);
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->d_lred, 0, sizeof(double) * B * 8, ctx->stream));
    // gs1 -> 0..2, gs2 -> 10..12, reductions (lam.s1, lam.s2, mu.s1, mu.s2)
    PM_LAUNCH(ctx, "lpt_adj_seed", launch_lpt_adj_seed(lr, np, B, ctx->d_fac, lam, mu, ctx->d_lred, ctx->stream));
    // S_bar = adjoint of s2 = IDFT(-i k / k^2 DFT S)
    PM_TRY(lat_r2c(ctx, 10, 3));
    PM_LAUNCH(ctx, "lpt_adj_second", launch_lpt_adj_second(lat_spec(ctx), 10, 9, ctx->stream));
    PM_TRY(lat_c2r(ctx, 9, 1));
    PM_LAUNCH(ctx, "lpt_adj_phi", launch_lpt_adj_phi(lr, np, B, ctx->stream));
    PM_TRY(lat_r2c(ctx, 0, 9));
    PM_LAUNCH(ctx, "noise", launch_noise(noise, seed, MeshRef{lat_field(ctx, 13), 0, ctx->lat_pad, lr.zs}, np, B,
                                ctx->stream));
    PM_TRY(lat_r2c(ctx, 13, 1));
    PM_LAUNCH(ctx, "lpt_adj_final", launch_lpt_adj_final(lat_spec(ctx), ctx->d_lin, 13, ctx->d_lred + 4 * B, ctx->stream));
    if (dnoise) {
        PM_TRY(lat_c2r(ctx, 0, 1));
        PM_LAUNCH(ctx, "unpad", launch_unpad(ctx->lat, ctx->lat_pad, lr.zs, dnoise, np, B, ctx->stream));
    }
    if (dcosmo) {
        std::vector<double> red((size_t)B * 8);
        PM_CUDA(ctx, cudaMemcpyAsync(red.data(), ctx->d_lred, sizeof(double) * red.size(), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        PM_TRY(device_check(ctx));  // a bounded TMA wait that timed out
        const double n3 = (double)np * np * np;
        for (int b = 0; b < B; ++b) {
            const HostTables &t = ctx->tabs[b];
            const double *g = red.data() + 4 * b;
            const double *pr = red.data() + 4 * B + 2 * b;
            double om = pr[1] / n3;
            for (int i = 0; i < 4; ++i) om += g[i] * t.dlpt[i];
            dcosmo[2 * b] = om;
            dcosmo[2 * b + 1] = pr[0] / n3 / ctx->s8[b];
        }
    }
    return PM_OK;
}

int pm_density(pm_ctx *ctx, const float *s, float *delta) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, delta, "delta"));
    DeviceGuard guard(ctx->device);
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    PaintArgs pa = paint_args(ctx, const_cast<float *>(s));
    pa.mesh = MeshRef{delta, 0, n3, ctx->P.n_m, 0};
    return paint_own(ctx, PAINT_DENSITY, pa, -1.f);  // delta = rho - 1
}

int pm_density_adjoint(pm_ctx *ctx, const float *s, const float *ddelta, float *ds) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, ddelta, "ddelta"));
    PM_TRY(check_ptr(ctx, ds, "ds"));
    DeviceGuard guard(ctx->device);
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    ReadArgs ra = read_args(ctx, const_cast<float *>(s));
    ra.mesh = MeshRef{const_cast<float *>(ddelta), 0, n3, ctx->P.n_m};
    ra.f = ds;
    PM_LAUNCH(ctx, read_kind(READ_GRAD), launch_read(READ_GRAD, ra, ctx->stream));
    return PM_OK;
}

int pm_mse_loss(pm_ctx *ctx, const float *s, const float *target, double *loss, float *dlds) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, target, "target"));
    if (!loss) return fail(ctx, PM_EINVAL, "loss must not be NULL");
    if (dlds) PM_TRY(check_ptr(ctx, dlds, "dlds"));
    DeviceGuard guard(ctx->device);
    const int B = ctx->P.n_batch;
    const MeshRef dref = density_ref(ctx);
    PM_TRY(paint_density(ctx, s, dref));
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->d_pk, 0, sizeof(double) * B, ctx->stream));
    PM_LAUNCH(ctx, "mse", launch_mse(dref, target, ctx->P.n_m, B, ctx->d_pk, ctx->stream));
    if (dlds) {
        ReadArgs ra = read_args(ctx, const_cast<float *>(s));
        ra.mesh = dref;
        ra.f = dlds;
        PM_LAUNCH(ctx, read_kind(READ_GRAD), launch_read(READ_GRAD, ra, ctx->stream));
    }
    std::vector<double> acc(B);
    PM_CUDA(ctx, cudaMemcpyAsync(acc.data(), ctx->d_pk, sizeof(double) * B, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PM_TRY(device_check(ctx));  // a bounded TMA wait that timed out
    const double n3 = std::pow((double)ctx->P.n_m, 3);
    for (int b = 0; b < B; ++b) loss[b] = acc[b] / n3;
    return PM_OK;
}

int pm_mesh_rfft(pm_ctx *ctx, const float *real, float *spec) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, real, "real"));
    PM_TRY(check_ptr(ctx, spec, "spec"));
    DeviceGuard guard(ctx->device);
    const int n = ctx->P.n_m, B = ctx->P.n_batch;
    if (ctx->own) {
        PM_TRY(own_forward(ctx, real, 1));
        PM_LAUNCH(ctx, "spec_copy", launch_spec_copy(ctx->spec, reinterpret_cast<float2 *>(spec), ctx->fg, true,
                                                     ctx->stream));
        return PM_OK;
    }
    const int zs = 2 * (n / 2 + 1);
    PM_CUDA(ctx, cudaMemcpy2DAsync(ctx->mesh, sizeof(float) * zs, real, sizeof(float) * n, sizeof(float) * n,
                                   (size_t)B * n * n, cudaMemcpyDeviceToDevice, ctx->stream));
    PM_TRY(mesh_r2c(ctx, 0, 1));
    PM_CUDA(ctx, cudaMemcpyAsync(spec, ctx->mesh, sizeof(float) * ctx->mesh_pad * B, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    return PM_OK;
}

int pm_mesh_irfft(pm_ctx *ctx, const float *spec, float *real) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, spec, "spec"));
    PM_TRY(check_ptr(ctx, real, "real"));
    DeviceGuard guard(ctx->device);
    const int n = ctx->P.n_m, B = ctx->P.n_batch;
    if (ctx->own) {
        PM_LAUNCH(ctx, "spec_copy", launch_spec_copy(ctx->spec, reinterpret_cast<float2 *>(const_cast<float *>(spec)),
                                                     ctx->fg, false, ctx->stream));
        return own_inverse(ctx, real, 1);
    }
    const int zs = 2 * (n / 2 + 1);
    PM_CUDA(ctx, cudaMemcpyAsync(ctx->mesh, spec, sizeof(float) * ctx->mesh_pad * B, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    PM_TRY(mesh_c2r(ctx, 0, 1));
    PM_CUDA(ctx, cudaMemcpy2DAsync(real, sizeof(float) * n, ctx->mesh, sizeof(float) * zs, sizeof(float) * n,
                                   (size_t)B * n * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return PM_OK;
}

int pm_power_spectrum(pm_ctx *ctx, const float *s, double *k_mean, double *power, double *n_modes) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    if (!k_mean || !power || !n_modes) return fail(ctx, PM_EINVAL, "host outputs must not be NULL");
    DeviceGuard guard(ctx->device);
    const int B = ctx->P.n_batch, nb = ctx->P.n_m / 2;
    const MeshRef dref = density_ref(ctx);
    PM_TRY(paint_density(ctx, s, dref));
    if (ctx->own)
        PM_TRY(own_forward(ctx, ctx->r1, 1));
    else
        PM_TRY(mesh_r2c(ctx, 0, 1));
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->d_pk, 0, sizeof(double) * B * 3 * nb, ctx->stream));
    PM_LAUNCH(ctx, "power_bins", launch_power_bins(mesh_spec(ctx), ctx->d_pk, nb, ctx->stream));
    std::vector<double> acc((size_t)B * 3 * nb);
    PM_CUDA(ctx, cudaMemcpyAsync(acc.data(), ctx->d_pk, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PM_TRY(device_check(ctx));  // a bounded TMA wait that timed out
    const double vol = std::pow(ctx->P.box, 3);
    const double n6 = std::pow((double)ctx->P.n_m, 6);
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < nb; ++i) {
            const double *a = acc.data() + ((size_t)b * nb + i) * 3;
            const double cnt = a[0] > 0 ? a[0] : 1.0;
            n_modes[(size_t)b * nb + i] = a[0];
            k_mean[(size_t)b * nb + i] = a[1] / cnt * (2.0 * M_PI / ctx->P.box);
            power[(size_t)b * nb + i] = vol / n6 * a[2] / cnt;
        }
    return PM_OK;
}

int pm_nn_param_count(void) { return nn_param_count(); }

int pm_nn_set_params(pm_ctx *ctx, const float *theta) {
    if (!ctx || !theta) return fail(ctx, PM_EINVAL, "ctx and theta must not be NULL");
    DeviceGuard guard(ctx->device);
    PM_TRY(ensure_nn(ctx));
    const int np = nn_param_count();
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PM_CUDA(ctx, cudaMemcpy(ctx->nn_theta, theta, sizeof(float) * np, cudaMemcpyHostToDevice));
    for (float *p : {ctx->nn_grad, ctx->nn_m, ctx->nn_v}) PM_CUDA(ctx, cudaMemset(p, 0, sizeof(float) * np));
    PM_LAUNCH(ctx, "nn_pack", launch_nn_pack(ctx->nn_theta, ctx->nnw, ctx->stream));
    return PM_OK;
}

int pm_nn_get_params(pm_ctx *ctx, float *theta, float *grad) {
    if (!ctx || (!theta && !grad)) return fail(ctx, PM_EINVAL, "nothing to copy");
    if (!ctx->nn_theta) return fail(ctx, PM_ESTATE, "no network parameters set");
    DeviceGuard guard(ctx->device);
    const int np = nn_param_count();
    PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PM_TRY(device_check(ctx));  // a bounded TMA wait that timed out
    if (theta) PM_CUDA(ctx, cudaMemcpy(theta, ctx->nn_theta, sizeof(float) * np, cudaMemcpyDeviceToHost));
    if (grad) PM_CUDA(ctx, cudaMemcpy(grad, ctx->nn_grad, sizeof(float) * np, cudaMemcpyDeviceToHost));
    return PM_OK;
}

int pm_nn_adam_step(pm_ctx *ctx, double lr, int64_t step) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    if (!ctx->nn_theta) return fail(ctx, PM_ESTATE, "no network parameters set");
    if (step < 1) return fail(ctx, PM_EINVAL, "Adam step count starts at 1");
    DeviceGuard guard(ctx->device);
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)step)));
    PM_LAUNCH(ctx, "adam", launch_adam(ctx->nn_theta, ctx->nn_grad, ctx->nn_m, ctx->nn_v, nn_param_count(), (float)lr,
                                       (float)b1, (float)b2, 1e-8f, c1, c2, ctx->stream));
    PM_LAUNCH(ctx, "nn_pack", launch_nn_pack(ctx->nn_theta, ctx->nnw, ctx->stream));
    return PM_OK;
}

int pm_nn_enable(pm_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    if (enable && !ctx->nn_theta) return fail(ctx, PM_ESTATE, "set the network parameters first");
    if (ctx->nn_err) {
        DeviceGuard guard(ctx->device);
        PM_TRY(nn_check(ctx));  // a time-out in the corrected integrations so far
    }
    ctx->nn_on = enable != 0;
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    return PM_OK;
}

int pm_nn_predict(pm_ctx *ctx, const float *s, double a, float *dF) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, dF, "dF"));
    if (!ctx->nn_theta) return fail(ctx, PM_ESTATE, "no network parameters set");
    DeviceGuard guard(ctx->device);
    PM_TRY(nn_forward_at(ctx, s, a, false));
    ReadArgs ra = read_args(ctx, const_cast<float *>(s));
    ra.f = dF;
    PM_TRY(read_forces(ctx, READ_FORCE, ra));
    return nn_check(ctx);
}

int pm_nn_train_step(pm_ctx *ctx, const float *s, const float *target, double a, double weight, double lr,
                     int64_t step, int apply, double *loss) {
    if (!ctx) return fail(nullptr, PM_EINVAL, "ctx must not be NULL");
    PM_TRY(check_ptr(ctx, s, "s"));
    PM_TRY(check_ptr(ctx, target, "target"));
    if (!ctx->nn_theta) return fail(ctx, PM_ESTATE, "no network parameters set");
    if (apply && step < 1) return fail(ctx, PM_EINVAL, "Adam step count starts at 1");
    if (!(weight > 0.0) || !std::isfinite(weight)) return fail(ctx, PM_EINVAL, "weight must be finite and > 0");
    DeviceGuard guard(ctx->device);
    const int np = nn_param_count();
    const int64_t parts = ctx->g.npart * ctx->P.n_batch;
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->nn_grad, 0, sizeof(float) * np, ctx->stream));
    PM_MEMSET(ctx, cudaMemsetAsync(ctx->nn_loss, 0, sizeof(double), ctx->stream));
    PM_TRY(nn_forward_at(ctx, s, a, true));
    // per-particle prediction, residual against the target, its cotangent
    ReadArgs ra = read_args(ctx, const_cast<float *>(s));
    ra.f = ctx->nn_part;
    PM_TRY(read_forces(ctx, READ_FORCE, ra));
    PM_LAUNCH(ctx, "nn_residual", launch_nn_residual(ctx->nn_part, target, 3 * parts, (float)(weight / parts),
                                                      ctx->nn_loss, ctx->stream));
    // adjoint of the read: paint the cotangent into slots 1..3 of a gradient mesh
    float *gmesh = reinterpret_cast<float *>(ctx->spec);
    const int64_t n3 = (int64_t)ctx->P.n_m * ctx->P.n_m * ctx->P.n_m;
    PM_MEMSET(ctx, cudaMemsetAsync(gmesh, 0, sizeof(float) * 4 * n3 * ctx->P.n_batch, ctx->stream));
    PaintArgs pa = paint_args(ctx, s, ctx->nn_part);
    pa.mesh = MeshRef{gmesh, 0, 4 * n3, ctx->P.n_m, 4};
    PM_LAUNCH(ctx, paint_kind(PAINT_ADJ), launch_paint(PAINT_ADJ, pa, ctx->stream));
    NNArgs na = nn_args(ctx, a);
    na.gmesh = gmesh;
    PM_LAUNCH(ctx, "nn_bwd", launch_nn_bwd(na, nn_cells(ctx), ctx->stream));
    if (apply) {
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)step)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)step)));
        PM_LAUNCH(ctx, "adam", launch_adam(ctx->nn_theta, ctx->nn_grad, ctx->nn_m, ctx->nn_v, np, (float)lr,
                                           (float)b1, (float)b2, 1e-8f, c1, c2, ctx->stream));
        PM_LAUNCH(ctx, "nn_pack", launch_nn_pack(ctx->nn_theta, ctx->nnw, ctx->stream));
    }
    if (loss) {
        double l = 0.0;
        PM_CUDA(ctx, cudaMemcpyAsync(&l, ctx->nn_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        PM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        *loss = l / (double)parts;
    }
    return PM_OK;
}

}  // extern "C"
