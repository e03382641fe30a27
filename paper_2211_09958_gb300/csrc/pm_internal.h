// Internal declarations of the GB300 PM library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pmgb {

// ------------------------------------------------------------ host side --

struct Params {
    int n_p, n_m, n_batch, n_steps;
    double box, a_init, a_final, h, n_s;
    int solver;  // PM_SOLVER_* bit mask
};

// Scale factor of step boundary n (0 .. n_steps) and of the half step
// after it: uniform in a (midpoint arithmetic) or, with the log-a solver
// flag (4), uniform in ln a (midpoint geometric).
double step_a(const Params &p, int n);
double half_step_a(const Params &p, int n);

struct Growth {
    double D1, dD1, D2, dD2, gp, gp2, gf;
};

struct HostTables {
    std::vector<double> ka, dr, kb;     // per step
    std::vector<double> dka, ddr, dkb;  // d/dOm
    double lpt[4];                      // D1, D2, g1, g2 at a_init
    double dlpt[4];                     // d/dOm
    double amp;                         // P(k) amplitude A
    double dlnamp;                      // d ln A / dOm
};

double hubble_e(double a, double om);
void growth_at(double om, const std::vector<double> &a, std::vector<Growth> *out);
// Growth-function emulator (growth_emulator.cpp): Omega_m in [0.1, 0.6],
// a in [1e-3, 1]; growth_emulated fills the same quantities as growth_at.
bool growth_emulator_covers(double om, double a);
void growth_emulate(double om, double a, double out[8]);
void growth_emulated(double om, const std::vector<double> &a, std::vector<Growth> *out);
void kdk_factors(double om, double a_init, double a_final, int n_steps, std::vector<double> *ka,
                 std::vector<double> *dr, std::vector<double> *kb);
void lpt_factors(double om, double a_init, double out[4], const Params *p = nullptr);
double bbks_transfer(double k, double om, double h);
double power_amplitude(double om, double s8, double h, double ns);
void host_tables(const Params &p, double om, double s8, HostTables *t);

// ---------------------------------------------------------- device side --

// Particle / mesh geometry shared by the particle kernels.
struct Geom {
    int np, nm, nb;      // particles per side, mesh per side, batch
    int64_t npart;       // np^3 particles per simulation
    int ratio;           // nm / np when it divides, else 0
    float inv_np;        // 1 / np
    float inv_h;         // nm / box
    float alpha;         // (nm / np)^3
    int order;           // assignment: 2 (CIC; also for 0) or 3 (TSC, solver flag 8)
};

// A set of real meshes: field f of batch b starts at ptr + f*fstride + b*bstride;
// rows along z are zs floats apart (zs = 2 (nm/2 + 1) for the cuFFT in-place
// layout, nm for a plain mesh).  il = 4: the four fields are interleaved per
// cell (cell c of run b at ptr + b*bstride + 4 c), fstride unused.
struct MeshRef {
    float *ptr;
    int64_t fstride, bstride;
    int zs;
    int il;
};

// Per step and simulation KDK factors on the device: x = K_a, y = Dr,
// z = K_b, w = K_a + K_b of the previous step (merged kick).
enum KickSel { KICK_A = 0, KICK_MERGED = 1, KICK_B = 2 };

enum PaintMode {
    PAINT_DENSITY = 0,   // paint weight alpha at s
    PAINT_ADJ = 2        // paint (alpha, mu_x, mu_y, mu_z) at s into 4 fields
};

struct PaintArgs {
    Geom g;
    const float *s;
    const float *mu;
    MeshRef mesh;
    int threads;  // block size: 128, 256 (also for 0) or 512 (autotuned)
};

// Particle-local work that precedes a force evaluation.
enum PreMode {
    PRE_KICK_DRIFT = 0,  // p += K_a f; s += Dr p            (first half of a KDK step)
    PRE_REV_DRIFT = 1    // s -= Dr p; mu += Dr lam; reduce lam.p (opens an adjoint step)
};

struct PreArgs {
    Geom g;
    float *s, *p;
    const float *f;
    const float *lam;
    float *mu;
    const float4 *table;
    int step;
    double *red;
    int red_bstride;
};

enum ReadMode {
    READ_FORCE = 0,       // f = F(s)
    READ_KICK_DRIFT = 1,  // p += c F; s += Dr p
    READ_HALF_KICK = 2,   // p += c F; f = F
    READ_ADJ = 3,         // F, vjp: lam += c vjp; p -= c F; reduce mu.F; optional fused reverse drift
    READ_GRAD = 4         // ds = alpha sum grad W mesh
};

struct ReadArgs {
    Geom g;
    float *s, *p, *f, *lam, *mu;
    MeshRef mesh;
    const float4 *table;
    int kick_step, kick_sel, drift_step;  // drift_step < 0: no drift
    double *red;          // kick reduction (batch stride red_bstride)
    int red_bstride;
    int red2_offset;      // drift reduction at red + red2_offset (0 when no drift)
    int threads;          // block size: 128, 256 (also for 0) or 512 (autotuned)
    // potential read (CIC, own-FFT meshes): when pot != NULL the force at each
    // corner is formed from the potential mesh by the 4-point difference
    // (pot [run][n^3] plain; the adjoint's psi one field later, at
    // pot + nb n^3) instead of being loaded from the float4 force mesh
    const float *pot;
    int lgn;              // log2 n_m
    float inv12h;         // 1 / (12 h)
    // when zero != NULL the read also clears zero4 float4 per run at
    // zero + b zero4 (the paint target of the next step, which the read no
    // longer needs), so that the next paint needs no separate zeroing pass
    float4 *zero;
    int64_t zero4;
};

cudaError_t launch_paint(int mode, const PaintArgs &a, cudaStream_t st);

// Binned, tile-owned CIC deposit (deposit_kernels.cu): particles binned by
// the DEPOSIT_TILE^3 tile of their base cell, then one block per column of
// tiles writes each owned mesh cell once; halo lines added by a second pass.
// Own-FFT plain meshes only (zs == n_m), n_m a multiple of DEPOSIT_TILE, CIC.
constexpr int DEPOSIT_TILE = 16;
struct DepositArgs {
    Geom g;
    const float *s, *mu;  // [run][npart][3]; mu for the 4-field paint
    int *key, *rank;      // [run * npart] tile and rank within it (bin_count)
    int *idx;             // [run * npart] particles in bin order (bin_scatter)
    int *count;           // [run * tiles] counters, zero between binnings
    int *offset;          // [run * tiles + 1] CSR offsets into idx
    int *chunk_sum;       // [deposit_scan_chunks] scan scratch
    float *mesh;          // plain [run][n^3] (1 field) or interleaved [run][n^3][4]
    float *halo;          // [run][nt][nt][2 TILE + 1][n_m] x fields halo lines
    int64_t tiles;        // tiles per run
    float base;           // value every cell starts from (added once, at the owned store)
};
bool deposit_supported(const Geom &g, int zs);
int64_t deposit_tiles(const Geom &g);
int64_t deposit_halo_floats(const Geom &g);  // for 4 fields
int64_t deposit_scan_chunks(const Geom &g);
cudaError_t deposit_prepare();  // kernel attributes; call once before any capture
cudaError_t launch_bin_count(const DepositArgs &a, cudaStream_t st);
cudaError_t launch_bin_scan_sums(const DepositArgs &a, cudaStream_t st);
cudaError_t launch_bin_scan(const DepositArgs &a, cudaStream_t st);
cudaError_t launch_bin_scatter(const DepositArgs &a, cudaStream_t st);
cudaError_t launch_deposit(int nf, const DepositArgs &a, cudaStream_t st);
cudaError_t launch_deposit_halo(int nf, const DepositArgs &a, cudaStream_t st);
cudaError_t launch_pre(int mode, const PreArgs &a, cudaStream_t st);
cudaError_t launch_read(int mode, const ReadArgs &a, cudaStream_t st);
cudaError_t launch_fill(float *ptr, int64_t n, float v, cudaStream_t st);
cudaError_t launch_unpad(const float *src, int64_t bstride, int zs, float *dst, int n, int nb, cudaStream_t st);
cudaError_t launch_mse(MeshRef mesh, const float *target, int n, int nb, double *acc, cudaStream_t st);
cudaError_t launch_kick(const Geom &g, float *p, const float *f, const float4 *table, int step, int sel,
                        float sign, cudaStream_t st);

// Spectral kernels over an rfft grid n x n x (n/2+1) (complex elements);
// field f of batch b starts at c + f*fstride + b*bstride.  blk = 0: rows
// [x][y][zc] with zc >= n/2+1; blk = 1: the own FFT's blocked layout
// [kz/8][x][y][kz%8] with zc/8 blocks.
struct Spec {
    float2 *c;
    int64_t fstride, bstride;
    int n, nb;
    float kf;  // 2 pi / box
    int zc;
    int blk;
    const float *grad;  // [n] 4-point difference gradient D(k) per axis index (force kernels)
    const float *dec;   // [n] per-axis CIC deconvolution 1/sinc^4(pi n_j / n), NULL = none
    int threads;        // force-kernel block size: 128, 256 (also for 0) or 512 (autotuned)
};

// The library's own FFT (fft_kernels.cu): spectra [field][run][kz/8][x][y][kz%8].
struct ZInvMap {
    CUtensorMap map;  // TMA descriptor of the blocked spectrum for one z-inverse block shape
    bool valid;
};

struct FftGeom {
    int n, nb, zc;
    int64_t fstride;    // complex elements per spectrum field (all runs)
    const float2 *tw;   // W_1024^j, j < 1024
    int zthreads;       // z-pass block size for n >= 256: 128, 256 (also for 0) or 512 (autotuned)
    int ztma;           // z inverse: 1 = stage the spectrum rows with TMA (where maps exist)
    int zstage;         // z forward (4 fields): 1 = coalesced 16-byte staging of the input rows
    const ZInvMap *tmaps;  // host array [3 output shapes: 4, 2, 1 slots][3 block sizes: 128, 256, 512], or NULL
    int *err;           // device flag set when a TMA wait times out
    int xwidth;         // x-pass pencil width in complex columns: 8 (also for 0) or 16 (autotuned)
};

struct PencilGeom {
    int64_t nkz, nmid, os, ms, ls;
};

bool own_fft_supported(int n);
int own_fft_zc(int n);
cudaError_t upload_fft_constants(float2 *tw_dev);
cudaError_t launch_fft_z_fwd(int g, const float *in, float2 *spec, const FftGeom &fg, cudaStream_t st);
constexpr int Z_INV_MAPS = 9;  // [output shape GO = 4, 2, 1][block size 128, 256, 512]
bool encode_z_inv_maps(float2 *spec, const FftGeom &fg, ZInvMap maps[Z_INV_MAPS]);
// gs = 4 or 3: spectrum fields -> 4-slot interleaved real mesh; gs = 2: two
// planar meshes (field 1 at out + nb n^3); gs = 1: plain real mesh.
cudaError_t launch_fft_z_inv(int gs, const float2 *spec, float *out, const FftGeom &fg, cudaStream_t st);
// Multipliers of the fused x round trip (launch_fft_xround): the spectral
// kernels' gradient and deconvolution tables, kf = 2 pi / box, the per-run
// prefactor (3/2) Om / n^3, and for the stencil form of the adjoint's psi
// 1 / (12 h) and whether the gradient is the 4-point difference.
struct XRoundArgs {
    float kf;
    const float *grad, *dec, *pref;
    float inv12h;  // 1 / (12 h): the 4-point difference stencil along x
    int fd;        // the gradient is the 4-point difference (not the spectral i k)
};
cudaError_t launch_fft_xround(bool adj, float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st);
// Potential form of the x round trip (4-point difference gradient only):
// nf = 1: field 0 (delta) -> field 0 (phi = IFFT(g delta), F_j = S_j phi);
// nf = 4: fields 0..3 (delta, u) -> 0 (phi), 1 (psi); nf = 2: fields 0
// (delta), 1 (v = sum_j S_j u_j) -> 0 (phi), 1 (psi = -IFFT(g v)).
cudaError_t launch_fft_xpot(int nf, float2 *spec, const FftGeom &fg, const XRoundArgs &xa, cudaStream_t st);
// F_j = S_j phi on the real mesh (the 4-point difference; symbol i D_j):
// in [gi][run][n^3] planar (phi, and psi for gi = 2) -> out [run][n^3]
// float4 (F_x, F_y, F_z, psi or 0).  n a power of two, >= 16.
cudaError_t launch_grad_stencil(const float *in, int gi, float4 *out, int n, int nb, float inv12h, cudaStream_t st);
// The adjoint source v = sum_j S_j u_j from the 4-field paint: in [run][n^3]
// float4 (rho, u_x, u_y, u_z) -> out [run][n^3] float2 (rho, v).  n a power
// of two, >= 16.
cudaError_t launch_vjp_source(const float4 *in, float2 *out, int n, int nb, float inv12h, cudaStream_t st);
cudaError_t launch_fft_pencils(int axis, bool inverse, float2 *spec, int f0, int nf, const FftGeom &fg,
                               cudaStream_t st);
cudaError_t launch_spec_copy(float2 *blocked, float2 *plain, const FftGeom &fg, bool to_plain, cudaStream_t st);

enum SpecMode { SPEC_FORCE = 0, SPEC_ADJ = 1 };
cudaError_t launch_spectral(int mode, const Spec &sp, const float *pref, cudaStream_t st);
cudaError_t launch_power_bins(const Spec &sp, double *acc, int nbins, cudaStream_t st);

// Initial conditions (lattice fields, same layout rules).
struct LinParams {
    double amp, om, h, ns, dlnamp, inv_vc;
};
cudaError_t launch_noise(const float *noise, uint64_t seed, MeshRef dst, int np, int nb, cudaStream_t st);
cudaError_t launch_lpt_linear(const Spec &sp, const LinParams *lp, cudaStream_t st);
cudaError_t launch_lpt_source(MeshRef lat, int np, int nb, int f_phi, int f_src, cudaStream_t st);
cudaError_t launch_lpt_second(const Spec &sp, int f_src, int f_out, float sign, cudaStream_t st);
cudaError_t launch_lpt_adj_second(const Spec &sp, int f_in, int f_out, cudaStream_t st);
cudaError_t launch_lpt_combine(MeshRef lat, int np, int nb, const float4 *fac, float *s, float *p, cudaStream_t st);
cudaError_t launch_lpt_adj_seed(MeshRef lat, int np, int nb, const float4 *fac, const float *lam, const float *mu,
                                double *red, cudaStream_t st);
cudaError_t launch_lpt_adj_phi(MeshRef lat, int np, int nb, cudaStream_t st);
cudaError_t launch_lpt_adj_final(const Spec &sp, const LinParams *lp, int f_noise, double *red, cudaStream_t st);

// ------------------------------------------------- learned correction ---

constexpr int NN_IN = 32, NN_HID = 128, NN_OUT = 3;

// Packed bf16 tensor-core (tcgen05) operands, K-major core-matrix layout
// (nn_cm_index), and FP32 biases (learned.cu):
//   forward  (rows = outputs, K = inputs)  w1c [128][32], w2c [128][128], w3c [16][128]
//   backward (rows = inputs, K = outputs)  w1b [32][128], w2b [128][128], w3b [128][16]
struct NNWeights {
    const __nv_bfloat16 *w1c, *w2c, *w3c, *w1b, *w2b, *w3b;
    const float *b1, *b2, *b3;
};
struct NNWeightsMut {
    __nv_bfloat16 *w1c, *w2c, *w3c, *w1b, *w2b, *w3b;
    float *b1, *b2, *b3;
};

// Element index of (row r, column k) of an R x K bf16 operand stored as
// 8 x 8 "core matrices" (8 rows of 16 contiguous bytes), K-direction core
// matrices R/8 * 128 bytes apart and row-direction ones 128 bytes apart: the
// no-swizzle K-major shared-memory layout the tcgen05 matrix descriptors
// address (leading byte offset R * 16, stride byte offset 128).
__host__ __device__ constexpr int nn_cm_index(int r, int k, int R) {
    return (((k >> 3) * (R >> 3) + (r >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}
struct NNArgs {
    NNWeights w;
    int n;               // mesh cells per side
    const float *rho;    // painted density [run][n^3] (alpha sum W), rho_stride floats per cell
    int rho_stride;      // 1 (plain mesh; also for 0) or 4 (slot 0 of the interleaved adjoint paint)
    float afeat;         // scale-factor feature
    const float *pref;   // per run 3/2 Om / n^3; output scale = pref * s_scale
    float s_scale;       // n^3 h, so that the output scale is 3/2 Om h
    float *out;          // interleaved 4-slot mesh [run][n^3][4], slots 0..2
    int accumulate;      // add to out instead of overwriting
    __nv_bfloat16 *xg, *h1g, *h2g, *g1g, *g2g, *g3g;  // training activations
    const float *gmesh;  // interleaved gradient mesh, slots 1..3
    float *grad, *gb1, *gb2, *gb3;
    int *err;            // set by the tensor-core kernel when a wait times out
    const __nv_bfloat16 *feat;  // [run][n^3] bf16(asinh(rho - 1)) (tensor-core path)
    // adjoint through the trajectory: the output cotangent is scaled per run
    // by the kick factor of table[kick_step * nb + run] (x: K_a, z: K_b, w:
    // merged; table NULL: 1), the feature cotangent g_x [cells][32] (FP32)
    // is written when gx != NULL
    const float4 *table;
    int kick_step, kick_sel, nb;
    float *gx;
};

#ifdef __CUDACC__
// The kick factor that scales run `run`'s output cotangent (1 without a table).
__device__ __forceinline__ float nn_kick_coef(const NNArgs &a, int64_t run) {
    if (!a.table) return 1.f;
    const float4 t = a.table[(int64_t)a.kick_step * a.nb + run];
    return a.kick_sel == KICK_A ? t.x : (a.kick_sel == KICK_B ? t.z : t.w);
}
#endif

int nn_param_count();
size_t nn_packed_bytes();
NNWeightsMut nn_carve(void *base);
cudaError_t launch_nn_pack(const float *theta, const NNWeightsMut &w, cudaStream_t st);
// Backward of one training step on the tensor cores: activation cotangents
// g3, g2, g1 (and the feature cotangent a.gx when set), bias gradients, then
// the weight gradients; needs the activations of the training forward.
cudaError_t launch_nn_bwd(const NNArgs &a, int64_t cells, cudaStream_t st);
// The weight gradients of one training step on the tensor cores (tcgen05):
// dW1 += x^T g1, dW2 += h1^T g2, dW3 += h2^T g3 over all cells.
cudaError_t launch_nn_wgrad_tc(const NNArgs &a, int64_t cells, cudaStream_t st);
cudaError_t nn_tc_prepare();
// bf16(asinh(rho - 1)) per cell; rho every `stride`-th float (1 or 4).
cudaError_t launch_nn_feat(const float *rho, __nv_bfloat16 *feat, int64_t cells, cudaStream_t st, int stride = 1);
// The network on the tensor cores (tcgen05) from the feature mesh a.feat;
// train = also store x, h1, h2 (a.xg, a.h1g, a.h2g) for the backward pass.
cudaError_t launch_nn_fwd_tc(const NNArgs &a, int64_t cells, cudaStream_t st, bool train = false);
cudaError_t launch_nn_residual(float *pred, const float *target, int64_t n, float scale, double *loss,
                               cudaStream_t st);
cudaError_t launch_adam(float *theta, float *grad, float *m, float *v, int np, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t st);
// g_rho(c) = sum_q g_x(c - o_q, q) / sqrt(1 + (rho(c) - 1)^2) / coef(run), written
// to slot 3 of the interleaved mesh out4; rho from slot 0 of rho4.
cudaError_t launch_nn_grad_rho(const NNArgs &a, const float *rho4, float *out4, int64_t cells, cudaStream_t st);
// dst[i] += src[i] over n float4 (the correction and density cotangent into
// the force / psi meshes).
cudaError_t launch_add4(float4 *dst, const float4 *src, int64_t n, cudaStream_t st);

}  // namespace pmgb
