// Binned, tile-owned CIC deposit: the density paint and the adjoint's
// 4-field paint without zeroing the mesh and without global float atomics.
//
// Paper (pmwd, arXiv:2211.09958), Summary: particle-mesh forces start from
// the mass assignment of the particles to the mesh; CIC weights W = product
// over axes of (1 - f, f) at the base cell c and c + 1 (mod n_m).  The sum
// is the same as the one-thread-per-particle scatter; only its order and
// the memory traffic differ.
//
// The mesh is cut into B^3 tiles (B = 16).  Every paint first bins the
// particles by the tile of their base cell (the cell `locate` gives, the
// same function the paint and the reads call):
//   bin_count    key = tile, rank within the tile from a warp-aggregated
//                atomic on the tile's counter (one atomic per distinct tile
//                in a warp: lattice-order warps span a few tiles);
//   bin_scan     exclusive prefix sum of the counters (two passes over
//                chunks of 4096) into the CSR offsets; zeroes the counters;
//   bin_scatter  idx[offset[key] + rank] = particle.
// The deposit gives each CTA one B x B column of tiles along z.  It walks
// the column's tiles in z order, adding each bin's particles into a
// shared-memory window of (B + 1)^3 cells with shared-memory atomics (the
// particles of a bin reach local cells 0 .. B along each axis).  After a
// tile it stores the B^3 owned cells to the mesh (each cell written once,
// plain coalesced stores), sends the x = B and y = B faces of the window to
// the column's halo lines, and keeps the z = B plane as the next tile's
// z = 0 plane (the window's planes rotate); the last tile's carry wraps
// onto the column's z = 0 cells.
// deposit_halo then adds each column's halo lines to the x = 0 and y = 0
// cells of the neighbouring columns (each cell updated by one thread, so
// the result does not depend on launch order).
// Traffic per paint, per field: the mesh written once, the halo lines
// (33 / 256 of the cells) written and read once, the x = 0 and y = 0 lines
// (31 / 256) read and written once, against zeroing plus an L2
// read-modify-write of every cell for the atomic scatter.  Measured at
// 512^3 particles on a 1024^3 mesh the binned form moves fewer bytes but
// runs slower (its per-tile phases are short and barrier-bound), so it is
// the alternative the tuner can pick, not the default.

#include "cic_common.cuh"

namespace pmgb {

namespace {

constexpr int B = DEPOSIT_TILE;   // cells per tile side
constexpr int W = B + 1;          // window side: the tile and its upper halo
constexpr int HL = 2 * B + 1;     // halo lines per column: x = B (y = 0 .. B), y = B (x = 0 .. B - 1)
constexpr int SCAN_CHUNK = 4096;  // counters per scan block (1024 threads x 4)

__device__ __forceinline__ int tile_of(const int c[3], int nt) {
    return ((c[0] / B) * nt + c[1] / B) * nt + c[2] / B;
}

__global__ void __launch_bounds__(256) k_bin_count(DepositArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.g.npart;
    const int nt = a.g.nm / B;
    int tile = 0;
    if (valid) {
        const int64_t gi = ((int64_t)b * a.g.npart + i) * 3;
        int c[3];
        float f[3];
        cic::locate(i, a.s[gi], a.s[gi + 1], a.s[gi + 2], a.g, c, f);
        tile = tile_of(c, nt);
    }
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const int lane = threadIdx.x & 31;
    const int64_t bin = (int64_t)b * a.tiles + tile;
    const unsigned peers = __match_any_sync(act, tile);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.count + bin, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t p = (int64_t)b * a.g.npart + i;
    a.key[p] = tile;
    a.rank[p] = base + __popc(peers & ((1u << lane) - 1u));
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the prefix and leaves the block total in *total.
__device__ __forceinline__ int block_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
        int ws = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        warp_sums[lane] = ws - w;  // exclusive prefix of the warp totals
        if (lane == 31) *total = ws;
    }
    __syncthreads();
    return warp_sums[warp] + x - v;
}

// Pass 1: the sum of each chunk of counters.
__global__ void __launch_bounds__(1024) k_bin_scan_sums(const int *count, int64_t n, int *chunk_sum) {
    __shared__ int ws[32];
    __shared__ int tot;
    const int64_t e0 = (int64_t)blockIdx.x * SCAN_CHUNK + 4 * threadIdx.x;
    int v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (e0 + q < n) v += count[e0 + q];
    block_scan(v, ws, &tot);
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
}

// Pass 2: offsets of the chunk (the sum of the earlier chunks' sums, then
// the chunk's own scan); zeroes the counters for the next binning.
__global__ void __launch_bounds__(1024) k_bin_scan(int *count, int64_t n, const int *chunk_sum, int *offset) {
    __shared__ int ws[32];
    __shared__ int tot;
    int pre = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) pre += chunk_sum[k];
    // block sum of pre (every thread adds the earlier chunks it read)
    const int before = block_scan(pre, ws, &tot);
    (void)before;
    const int chunk_base = tot;
    __syncthreads();
    const int64_t e0 = (int64_t)blockIdx.x * SCAN_CHUNK + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = e0 + q < n ? count[e0 + q] : 0;
    const int x = block_scan(v[0] + v[1] + v[2] + v[3], ws, &tot);
    int run = chunk_base + x;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (e0 + q < n) {
            offset[e0 + q] = run;
            run += v[q];
            count[e0 + q] = 0;
        }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) offset[n] = run;
}

__global__ void __launch_bounds__(256) k_bin_scatter(DepositArgs a) {
    const int b = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.g.npart) return;
    const int64_t p = (int64_t)b * a.g.npart + i;
    const int64_t pos = (int64_t)a.offset[(int64_t)b * a.tiles + a.key[p]] + a.rank[p];
    if (pos >= 0 && pos < a.g.npart * a.g.nb) a.idx[pos] = (int)i;  // always true when the counters started at zero
}

// One particle's inputs: lattice index (-1: none), displacement, and for
// the 4-field paint its mu.
template <int NF>
struct Part {
    int i;
    float s[3];
    float m[NF == 4 ? 3 : 1];
};

template <int NF>
__device__ __forceinline__ Part<NF> load_part(int i, const float *s, const float *mu, int64_t npart) {
    Part<NF> r;
    r.i = (i >= 0 && i < npart) ? i : -1;  // out of range only for an inconsistent binning
    if (r.i < 0) {
        r.s[0] = r.s[1] = r.s[2] = 0.f;
        if (NF == 4) r.m[0] = r.m[1] = r.m[2] = 0.f;
        return r;
    }
    const float *sp = s + (int64_t)r.i * 3;
    r.s[0] = sp[0];
    r.s[1] = sp[1];
    r.s[2] = sp[2];
    if (NF == 4) {
        const float *mp = mu + (int64_t)r.i * 3;
        r.m[0] = mp[0];
        r.m[1] = mp[1];
        r.m[2] = mp[2];
    }
    return r;
}

// The CIC corners of the particles of one warp iteration into the window
// (field-major: field q of cell (x, y, physical plane zp) at
// q W^3 + (x W + y) W + zp).  Lanes whose particles share a base cell are
// merged first: the lowest lane of each such group collects the others'
// fractions and values by shuffles and adds the group's corner sums with
// one shared-memory atomic each, so that a dense cell costs one atomic per
// corner instead of one per particle and corner (same-address atomics of a
// warp serialise).  The corners go in two halves (x offset 0, then 1) to
// bound the registers.  Every lane of the warp iteration calls this; lanes
// without a particle (p.i < 0) join the shuffles only.
template <int NF>
__device__ __forceinline__ void deposit_group(float *win, const Part<NF> &p, const Geom &g, int tx, int ty, int kz,
                                              int zbase) {
    constexpr int W3 = W * W * W;
    const int lane = threadIdx.x & 31;
    int c[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    if (p.i >= 0) cic::locate(p.i, p.s[0], p.s[1], p.s[2], g, c, f);
    const float wv[4] = {g.alpha, NF == 4 ? p.m[0] : 0.f, NF == 4 ? p.m[NF == 4 ? 1 : 0] : 0.f,
                         NF == 4 ? p.m[NF == 4 ? 2 : 0] : 0.f};
    const int lx = c[0] - tx * B, ly = c[1] - ty * B, lz = c[2] - kz * B;  // 0 .. B - 1
    const bool valid = p.i >= 0 && (unsigned)lx < B && (unsigned)ly < B && (unsigned)lz < B;
    const int key = valid ? (lx * B + ly) * B + lz : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);  // the callers keep whole warps together
    const bool lead = valid && lane == __ffs(peers) - 1;
    int z0 = zbase + lz;
    if (z0 >= W) z0 -= W;
    const int z1 = z0 + 1 == W ? 0 : z0 + 1;
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) {
        const float wx = ox ? f[0] : 1.f - f[0];
        float acc[4][NF];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float w = wx * ((k & 2) ? f[1] : 1.f - f[1]) * ((k & 1) ? f[2] : 1.f - f[2]);
#pragma unroll
            for (int q = 0; q < NF; ++q) acc[k][q] = w * wv[q];
        }
        unsigned rest = peers & (peers - 1);  // the group's other lanes, lowest first
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            float gf[3], gv[NF];
#pragma unroll
            for (int t = 0; t < 3; ++t) gf[t] = __shfl_sync(peers, f[t], src);
#pragma unroll
            for (int q = 0; q < NF; ++q) gv[q] = __shfl_sync(peers, wv[q], src);
            const float gx = ox ? gf[0] : 1.f - gf[0];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float w = gx * ((k & 2) ? gf[1] : 1.f - gf[1]) * ((k & 1) ? gf[2] : 1.f - gf[2]);
#pragma unroll
                for (int q = 0; q < NF; ++q) acc[k][q] += w * gv[q];
            }
        }
        if (lead) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int cell = ((lx + ox) * W + (ly + (k >> 1))) * W + ((k & 1) ? z1 : z0);
#pragma unroll
                for (int q = 0; q < NF; ++q) atomicAdd(win + q * W3 + cell, acc[k][q]);
            }
        }
    }
}

// NF = 1: the density (weight alpha) into a plain mesh [run][n^3];
// NF = 4: (alpha, mu_x, mu_y, mu_z) into the interleaved mesh [run][n^3][4].
// The window's z planes rotate: local plane z of the current tile is the
// physical plane (zbase + z) mod W, and zbase advances by B per tile, so the
// carried plane (local B) becomes the next tile's local 0 in place; the
// store loops clear each plane they read, which leaves the next tile's
// planes 1 .. B zero.  The particle loads run ahead of the tiles: a
// thread's first PER particles of tile k + 1 are loaded while tile k is
// deposited and stored, their bin entries two tiles ahead (the column's bin
// offsets sit in shared memory); larger bins load the rest in place.
template <int NF, int T>
__global__ void __launch_bounds__(T, NF == 4 ? 2 : 4) k_deposit(DepositArgs a) {
    constexpr int W3 = W * W * W;
    constexpr int PER = NF == 4 ? 1 : 2;
    extern __shared__ float4 win4[];
    float *win = reinterpret_cast<float *>(win4);  // [NF][W][W][W]
    int *soff = reinterpret_cast<int *>(win + NF * W3);  // [nt + 1] bin offsets of this column
    const int nm = a.g.nm, nt = nm / B, b = blockIdx.y;
    const int tx = blockIdx.x / nt, ty = blockIdx.x % nt;
    const int64_t n3 = (int64_t)nm * nm * nm;
    const int64_t col = ((int64_t)b * nt + tx) * nt + ty;  // this column's halo lines
    const int64_t total = a.g.npart * a.g.nb;
    float *mesh = a.mesh + (int64_t)b * n3 * NF;
    float *halo = a.halo + col * HL * nm * NF;
    const float *s = a.s + (int64_t)b * a.g.npart * 3;
    const float *mu = NF == 4 ? a.mu + (int64_t)b * a.g.npart * 3 : nullptr;
    const int64_t bin0 = (int64_t)b * a.tiles + ((int64_t)tx * nt + ty) * nt;
    for (int e = threadIdx.x; e < NF * W3; e += T) win[e] = 0.f;
    for (int k = threadIdx.x; k <= nt; k += T) soff[k] = (int)min(max((int64_t)a.offset[bin0 + k], (int64_t)0), total);
    __syncthreads();
    auto entry = [&](int k, int u) -> int {  // bin entry u of this thread in tile k, or -1
        if (k >= nt) return -1;
        const int j = soff[k] + threadIdx.x + u * T;
        return j < soff[k + 1] ? a.idx[j] : -1;
    };
    Part<NF> nxt[PER];
    int ent[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) nxt[u] = load_part<NF>(entry(0, u), s, mu, a.g.npart);
#pragma unroll
    for (int u = 0; u < PER; ++u) ent[u] = entry(1, u);
    int zbase = 0;
    for (int kz = 0; kz < nt; ++kz) {
        Part<NF> cur[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            cur[u] = nxt[u];
            nxt[u] = load_part<NF>(ent[u], s, mu, a.g.npart);  // tile kz + 1, used next iteration
            ent[u] = entry(kz + 2, u);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u)
            if (soff[kz] + (int)threadIdx.x - (int)(threadIdx.x & 31) + u * T < soff[kz + 1])  // warp has work
                deposit_group<NF>(win, cur[u], a.g, tx, ty, kz, zbase);
        for (int j = soff[kz] + threadIdx.x + PER * T; j - (int)(threadIdx.x & 31) < soff[kz + 1]; j += T) {
            const Part<NF> p = load_part<NF>(j < soff[kz + 1] ? a.idx[j] : -1, s, mu, a.g.npart);
            deposit_group<NF>(win, p, a.g, tx, ty, kz, zbase);
        }
        __syncthreads();
        // the owned cells, z fastest (B consecutive cells of a row per B threads),
        // each cleared as it is read
        for (int e = threadIdx.x; e < B * B * B; e += T) {
            const int x = e / (B * B), y = (e / B) % B, z = e % B;
            int zp = zbase + z;
            if (zp >= W) zp -= W;
            const int w = ((x * W) + y) * W + zp;
            const int64_t g = ((int64_t)(tx * B + x) * nm + (ty * B + y)) * nm + kz * B + z;
            if (NF == 4) {
                const float4 v = make_float4(win[w] + a.base, win[W3 + w] + a.base, win[2 * W3 + w] + a.base,
                                             win[3 * W3 + w] + a.base);
                reinterpret_cast<float4 *>(mesh)[g] = v;
            } else {
                mesh[g] = win[w] + a.base;
            }
#pragma unroll
            for (int q = 0; q < NF; ++q) win[q * W3 + w] = 0.f;
        }
        // halo lines: h < B + 1 -> (x = B, y = h); h > B -> (x = h - B - 1, y = B)
        for (int e = threadIdx.x; e < HL * B; e += T) {
            const int h = e / B, z = e % B;
            const int x = h <= B ? B : h - B - 1, y = h <= B ? h : B;
            int zp = zbase + z;
            if (zp >= W) zp -= W;
            const int w = ((x * W) + y) * W + zp;
            const int64_t o = (int64_t)h * nm + kz * B + z;
            if (NF == 4)
                reinterpret_cast<float4 *>(halo)[o] = make_float4(win[w], win[W3 + w], win[2 * W3 + w], win[3 * W3 + w]);
            else
                halo[o] = win[w];
#pragma unroll
            for (int q = 0; q < NF; ++q) win[q * W3 + w] = 0.f;
        }
        zbase = zbase + B >= W ? zbase + B - W : zbase + B;  // the carried plane is local 0 now
        __syncthreads();
    }
    // the last tile's carry belongs to z = 0 (periodic): add it to the owned
    // z = 0 cells and the z = 0 halo entries this block stored in its first tile
    for (int e = threadIdx.x; e < W * W; e += T) {
        const int x = e / W, y = e % W;
        const int w = e * W + zbase;
        float *dst;
        if (x < B && y < B)
            dst = mesh + (((int64_t)(tx * B + x) * nm + (ty * B + y)) * nm) * NF;
        else
            dst = halo + (int64_t)(x == B ? y : B + 1 + x) * nm * NF;
#pragma unroll
        for (int q = 0; q < NF; ++q) dst[q] += win[q * W3 + w];
    }
}

// Adds the halo lines of the columns at (tx - 1, ty), (tx, ty - 1) and
// (tx - 1, ty - 1) (periodic) to this column's x = 0 and y = 0 cells.
template <int NF>
__global__ void __launch_bounds__(256) k_deposit_halo(DepositArgs a) {
    const int nm = a.g.nm, nt = nm / B, b = blockIdx.y;
    const int tx = blockIdx.x / nt, ty = blockIdx.x % nt;
    const int xm = (tx + nt - 1) % nt, ym = (ty + nt - 1) % nt;
    const int64_t n3 = (int64_t)nm * nm * nm;
    const int64_t line = (int64_t)HL * nm * NF;
    const float *hx = a.halo + (((int64_t)b * nt + xm) * nt + ty) * line;  // x = B lines of (tx - 1, ty)
    const float *hy = a.halo + (((int64_t)b * nt + tx) * nt + ym) * line;  // y = B lines of (tx, ty - 1)
    const float *hxy = a.halo + (((int64_t)b * nt + xm) * nt + ym) * line; // corner line of (tx - 1, ty - 1)
    float *mesh = a.mesh + (int64_t)b * n3 * NF;
    for (int64_t e = threadIdx.x; e < (int64_t)(2 * B - 1) * nm; e += blockDim.x) {
        const int l = (int)(e / nm), z = (int)(e % nm);
        // l < B: cell (0, l); l >= B: cell (l - B + 1, 0)
        const int x = l < B ? 0 : l - B + 1, y = l < B ? l : 0;
        float add[NF];
        const int64_t o = (int64_t)z * NF;
        if (x == 0) {
#pragma unroll
            for (int q = 0; q < NF; ++q) add[q] = hx[(int64_t)y * nm * NF + o + q];
            if (y == 0)
#pragma unroll
                for (int q = 0; q < NF; ++q)
                    add[q] += hy[(int64_t)(B + 1) * nm * NF + o + q] + hxy[(int64_t)B * nm * NF + o + q];
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) add[q] = hy[(int64_t)(B + 1 + x) * nm * NF + o + q];
        }
        float *dst = mesh + (((int64_t)(tx * B + x) * nm + (ty * B + y)) * nm + z) * NF;
#pragma unroll
        for (int q = 0; q < NF; ++q) dst[q] += add[q];
    }
}

// block sizes: 256 threads for the 19.6 KB density window (8 blocks an
// SM), 512 for the 78.6 KB four-field window (2 blocks an SM)
template <int NF>
constexpr int deposit_threads() {
    return NF == 4 ? 512 : 256;
}

// the window, then the column's bin offsets (n_m <= 4096: at most 257)
template <int NF>
constexpr int deposit_smem() {
    return W * W * W * NF * (int)sizeof(float) + 4 * (4096 / B + 1);
}

}  // namespace

bool deposit_supported(const Geom &g, int zs) {
    // CSR offsets are 32-bit: at most 2^31 - 1 particles over the batch
    return g.order != 3 && g.nm % B == 0 && g.nm <= 4096 && zs == g.nm && g.npart * g.nb < ((int64_t)1 << 31);
}

int64_t deposit_tiles(const Geom &g) {
    const int64_t nt = g.nm / B;
    return nt * nt * nt;
}

int64_t deposit_halo_floats(const Geom &g) {
    const int64_t nt = g.nm / B;
    return (int64_t)g.nb * nt * nt * HL * g.nm * 4;
}

int64_t deposit_scan_chunks(const Geom &g) {
    return (deposit_tiles(g) * g.nb + SCAN_CHUNK - 1) / SCAN_CHUNK;
}

cudaError_t deposit_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_deposit<4, deposit_threads<4>()>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, deposit_smem<4>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_deposit<1, deposit_threads<1>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                deposit_smem<1>());
}

cudaError_t launch_bin_count(const DepositArgs &a, cudaStream_t st) {
    k_bin_count<<<dim3((unsigned)((a.g.npart + 255) / 256), a.g.nb), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bin_scan_sums(const DepositArgs &a, cudaStream_t st) {
    const int64_t n = a.tiles * a.g.nb;
    k_bin_scan_sums<<<(unsigned)((n + SCAN_CHUNK - 1) / SCAN_CHUNK), 1024, 0, st>>>(a.count, n, a.chunk_sum);
    return cudaGetLastError();
}

cudaError_t launch_bin_scan(const DepositArgs &a, cudaStream_t st) {
    const int64_t n = a.tiles * a.g.nb;
    k_bin_scan<<<(unsigned)((n + SCAN_CHUNK - 1) / SCAN_CHUNK), 1024, 0, st>>>(a.count, n, a.chunk_sum, a.offset);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const DepositArgs &a, cudaStream_t st) {
    k_bin_scatter<<<dim3((unsigned)((a.g.npart + 255) / 256), a.g.nb), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_deposit(int nf, const DepositArgs &a, cudaStream_t st) {
    const int nt = a.g.nm / B;
    const dim3 grid((unsigned)(nt * nt), a.g.nb);
    if (nf == 4)
        k_deposit<4, deposit_threads<4>()><<<grid, deposit_threads<4>(), deposit_smem<4>(), st>>>(a);
    else
        k_deposit<1, deposit_threads<1>()><<<grid, deposit_threads<1>(), deposit_smem<1>(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_deposit_halo(int nf, const DepositArgs &a, cudaStream_t st) {
    const int nt = a.g.nm / B;
    const dim3 grid((unsigned)(nt * nt), a.g.nb);
    if (nf == 4)
        k_deposit_halo<4><<<grid, 256, 0, st>>>(a);
    else
        k_deposit_halo<1><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pmgb
