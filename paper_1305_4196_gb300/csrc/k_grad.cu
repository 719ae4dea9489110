// k_grad.cu - reverse-mode derivatives of the Lennard-Jones forces (force matching).
//
// For a scalar loss L of the forces with G = dL/dF given, the chain rule over the
// pairs inside their cutoffs (the pair set held fixed: the cutoff contributes no
// derivative) gives, per pair (i, j) with d = x_i - x_j, f_ij = g(r^2) d and
// w = G_i - G_j:
//     dL/dx_i += g w + 2 g' (w . d) d          (and the negative on x_j)
//     dL/deps_ab += (w . d) g / eps
//     dL/dsig_ab += (w . d) * 144 eps (4 s6^2 - s6) / (sig r^2)
// with s6 = (sig^2/r^2)^3, g = 24 eps (2 s6^2 - s6) / r^2 and
// g' = dg/d(r^2) = 24 eps (4 s6 - 14 s6^2) / r^4.  The energy's parameter
// derivatives, dE/deps_ab = sum 4 (s6^2 - s6) and dE/dsig_ab = sum 24 eps
// (2 s6^2 - s6) / sig, come from the same pass.
//
// The kernel follows the full-list force kernels: one CTA per 2x2x2-cell block with
// the block's 4x4x4-cell tile (coordinates, species and global index) in shared
// memory, G read from the cell-ordered global copy (L2-resident); one thread per
// atom accumulating only its own dL/dx_i (each pair is seen from both sides, which
// also gives the negative term on x_j).  Parameter terms are accumulated per atom by
// neighbour species and summed in a fixed order afterwards, so every result is
// deterministic.  T = double on FP64 systems, float (FP32 pair arithmetic,
// block-frame coordinates) on mixed-precision ones.
#include "tile.cuh"

#include <algorithm>

namespace mdgb {

constexpr int G_THREADS = 128;
static int g_sm_count = 0;  // SMs of the device, read at initialisation
constexpr int G_QUANT = 4;  // per species pair: dL/deps, dL/dsig, dE/deps, dE/dsig

template <typename T>
struct GradTile {
    T *x, *y, *z;
    int *sp, *gid;  // species, cell-ordered global index (the dummy slot: -1)
};

// Global index of every tile atom, one warp per tile cell.
__device__ __forceinline__ void stage_gid(const TileMeta& m, int* __restrict__ gid) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int slot = warp; slot < 64; slot += nw) {
        const int u0 = m.prefix[slot], cnt = m.prefix[slot + 1] - u0, j0 = m.start[slot];
        for (int e = lane; e < cnt; e += 32) gid[u0 + e] = j0 + e;
    }
}

__device__ __forceinline__ void add_by_species(double (&P)[MAX_SPECIES][G_QUANT], int sj, int q, double v) {
    // explicit branches keep the accumulators in registers
    if (sj == 0) P[0][q] += v;
    else if (sj == 1) P[1][q] += v;
    else if (sj == 2) P[2][q] += v;
    else P[3][q] += v;
}

// prm: n x (nsp*nsp*G_QUANT), row i holds atom i's terms in the columns of its own
// species row (t = s_i * nsp + s_j), zero elsewhere; each unordered pair is visited
// from both sides, so every term is halved.
template <typename T>
__global__ void __launch_bounds__(G_THREADS) k_force_backward(DevState s, Geometry g, PairTable pt, TileOffsets to,
                                                              int tile_cap, const double* __restrict__ G,
                                                              double* __restrict__ gx_out, double* __restrict__ prm,
                                                              int want_energy, int split) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    // split CTAs share one block: each stages the whole tile and takes every split-th group
    // of G_THREADS own atoms, so that a small system still spreads over the SMs
    const int b = spatial_block(g, blockIdx.x / split), part = blockIdx.x % split;
    tile_meta(g, s.cell_start, b, m);
    const int T_ = m.prefix[64];
    if (T_ + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    const int nown = m.prefix[8];
    if (nown == 0) return;
    GradTile<T> t;
    t.x = reinterpret_cast<T*>(smem);
    t.y = t.x + tile_cap;
    t.z = t.y + tile_cap;
    t.sp = reinterpret_cast<int*>(t.z + tile_cap);
    t.gid = t.sp + tile_cap;
    if constexpr (sizeof(T) == 8) {
        tile_stage_f64(s, g, m, b, t.x, t.y, t.z, t.sp);
    } else {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int slot = warp; slot < 64; slot += nw) {
            const int c = c_tiles.coord_of_idx[slot];
            const float ox = pick4(to.off[0], c & 3), oy = pick4(to.off[1], (c >> 2) & 3),
                        oz = pick4(to.off[2], c >> 4);
            const int u0 = m.prefix[slot], cnt = m.prefix[slot + 1] - u0, j0 = m.start[slot];
            for (int e = lane; e < cnt; e += 32) {
                const float4 p = s.xr[j0 + e];
                t.x[u0 + e] = p.x + ox;
                t.y[u0 + e] = p.y + oy;
                t.z[u0 + e] = p.z + oz;
                t.sp[u0 + e] = __float_as_int(p.w);
            }
        }
        if (threadIdx.x == 0) {
            t.x[T_] = t.y[T_] = t.z[T_] = 1.0e4f;
            t.sp[T_] = 0;
        }
    }
    stage_gid(m, t.gid);
    if (threadIdx.x == 0) t.gid[T_] = -1;
    __syncthreads();
    const int nsp = pt.nsp;
    const int ncol = nsp * nsp * G_QUANT;
    const int blk0 = m.start[0];
    const int64_t n = s.n;
    for (int ui = part * blockDim.x + threadIdx.x; ui < nown; ui += split * blockDim.x) {
        const int64_t gi = blk0 + ui;
        const T xi = t.x[ui], yi = t.y[ui], zi = t.z[ui];
        const T Gx = G ? (T)G[gi] : T(0), Gy = G ? (T)G[n + gi] : T(0), Gz = G ? (T)G[2 * n + gi] : T(0);
        const int si = t.sp[ui];
        T ax = 0, ay = 0, az = 0;
        double P[MAX_SPECIES][G_QUANT] = {};
        const int cnt = s.nl_cnt[gi];
        for (int k = 0; k < cnt; ++k) {
            const int u = s.nl[((size_t)(k >> 3) * s.np + gi) * 8 + (k & 7)];
            const T dx = xi - t.x[u], dy = yi - t.y[u], dz = zi - t.z[u];
            const T r2 = dx * dx + dy * dy + dz * dz;
            const int sj = t.sp[u];
            const int tt = si * nsp + sj;
            if (sizeof(T) == 8) {
                if (!(r2 < (T)pt.rc2_d[tt])) continue;
            } else {
                if (!((float)r2 < pt.rc2hi_f[tt])) continue;
                if (!((float)r2 < pt.rc2lo_f[tt]) &&  // rare: decide the cutoff in FP64
                    !fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], (int)gi, t.gid[u], pt.rc2_d[tt]))
                    continue;
            }
            const T sig2 = sizeof(T) == 8 ? (T)pt.sig2_d[tt] : (T)pt.sig2_f[tt];
            const T e = sizeof(T) == 8 ? (T)pt.eps_d[tt] : (T)(pt.c4_f[tt] * 0.25f);
            const T sig = (T)pt.sig_d[tt];
            const T inv = T(1) / r2;
            const T sr2 = sig2 * inv;
            const T s6 = sr2 * sr2 * sr2;
            const T gq = T(24) * e * (T(2) * s6 * s6 - s6) * inv;
            const T gp = T(24) * e * (T(4) * s6 - T(14) * s6 * s6) * inv * inv;
            const int gj = t.gid[u];
            const T wx = Gx - (G ? (T)G[gj] : T(0)), wy = Gy - (G ? (T)G[n + gj] : T(0)),
                    wz = Gz - (G ? (T)G[2 * n + gj] : T(0));
            const T wd = wx * dx + wy * dy + wz * dz;
            const T two_gp_wd = T(2) * gp * wd;
            ax += gq * wx + two_gp_wd * dx;
            ay += gq * wy + two_gp_wd * dy;
            az += gq * wz + two_gp_wd * dz;
            add_by_species(P, sj, 0, (double)(wd * (T(24) * (T(2) * s6 * s6 - s6) * inv)));
            add_by_species(P, sj, 1, (double)(wd * (T(144) * e * (T(4) * s6 * s6 - s6) * inv / sig)));
            if (want_energy) {
                add_by_species(P, sj, 2, (double)(T(4) * (s6 * s6 - s6)));
                add_by_species(P, sj, 3, (double)(T(24) * e * (T(2) * s6 * s6 - s6) / sig));
            }
        }
        if (gx_out) {
            gx_out[gi] = (double)ax;
            gx_out[n + gi] = (double)ay;
            gx_out[2 * n + gi] = (double)az;
        }
        double* row = prm + gi * ncol;
        for (int c = 0; c < ncol; ++c) row[c] = 0.0;
#pragma unroll
        for (int b2 = 0; b2 < MAX_SPECIES; ++b2) {
            if (b2 >= nsp) break;
#pragma unroll
            for (int q = 0; q < G_QUANT; ++q) row[(si * nsp + b2) * G_QUANT + q] = 0.5 * P[b2][q];
        }
    }
}

// Column sums of an n x ncol matrix in a fixed order: per-CTA partials over contiguous
// row ranges, then one CTA over the partials.
constexpr int CS_THREADS = 256;

__global__ void __launch_bounds__(CS_THREADS) k_colsum_partials(const double* __restrict__ a, int64_t n, int ncol,
                                                                int64_t chunk, double* __restrict__ part) {
    __shared__ double sh[CS_THREADS];
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    for (int c = 0; c < ncol; ++c) {
        double acc = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += CS_THREADS) acc += a[i * ncol + c];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = CS_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * ncol + c] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CS_THREADS) k_colsum_final(const double* __restrict__ part, int nparts, int ncol,
                                                             double* __restrict__ out) {
    __shared__ double sh[CS_THREADS];
    for (int c = 0; c < ncol; ++c) {
        double acc = 0.0;
        for (int p = threadIdx.x; p < nparts; p += CS_THREADS) acc += part[p * ncol + c];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = CS_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sh[0];
        __syncthreads();
    }
}

// G (N x 3, original order) -> cell order, 3 x n
__global__ void k_grad_in(DevState s, const double* __restrict__ G, double* __restrict__ Gc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t o = s.orig[i];
    Gc[i] = G[3 * o];
    Gc[s.n + i] = G[3 * o + 1];
    Gc[2 * s.n + i] = G[3 * o + 2];
}

// cell order, 3 x n -> original order, N x 3
__global__ void k_grad_out(DevState s, const double* __restrict__ gc, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t o = s.orig[i];
    out[3 * o] = gc[i];
    out[3 * o + 1] = gc[s.n + i];
    out[3 * o + 2] = gc[2 * s.n + i];
}

size_t backward_smem_bytes(int fp64, int tile_cap) {
    return (size_t)tile_cap * (3 * (fp64 ? sizeof(double) : sizeof(float)) + 2 * sizeof(int));
}

size_t backward_scratch_doubles(int64_t n, int nsp, int nparts) {
    return 3 * (size_t)n + 3 * (size_t)n + (size_t)n * nsp * nsp * G_QUANT + (size_t)nparts * nsp * nsp * G_QUANT +
           (size_t)nsp * nsp * G_QUANT;
}

// scratch layout: Gc (3n) | gx (3n) | prm (n x ncol) | partials (nparts x ncol) | totals (ncol)
void launch_force_backward(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                           int tile_cap, int fp64, const double* G, double* gx_orig, int want_energy,
                           double* scratch, int nparts, cudaStream_t st) {
    const int64_t n = s.n;
    const int ncol = pt.nsp * pt.nsp * G_QUANT;
    double* Gc = scratch;
    double* gxc = Gc + 3 * n;
    double* prm = gxc + 3 * n;
    double* part = prm + (size_t)n * ncol;
    double* tot = part + (size_t)nparts * ncol;
    const int bs = 256;
    const unsigned nb = (unsigned)((n + bs - 1) / bs);
    if (G) k_grad_in<<<nb, bs, 0, st>>>(s, G, Gc);
    const size_t smem = backward_smem_bytes(fp64, tile_cap);
    // CTAs per block: enough for about one own atom per thread, while the grid is below two
    // CTAs per SM (small systems, e.g. force-matching snapshots of a few 10^4 atoms)
    const int sms = g_sm_count > 0 ? g_sm_count : 152;
    const int64_t per_block = (n + g.nblock - 1) / g.nblock;
    int split = (int)std::min<int64_t>((per_block + G_THREADS - 1) / G_THREADS, (2 * sms + g.nblock - 1) / g.nblock);
    split = std::max(1, std::min(split, 8));
    const unsigned grid = (unsigned)g.nblock * (unsigned)split;
    if (fp64)
        k_force_backward<double><<<grid, G_THREADS, smem, st>>>(s, g, pt, to, tile_cap, G ? Gc : nullptr,
                                                               gx_orig ? gxc : nullptr, prm, want_energy, split);
    else
        k_force_backward<float><<<grid, G_THREADS, smem, st>>>(s, g, pt, to, tile_cap, G ? Gc : nullptr,
                                                              gx_orig ? gxc : nullptr, prm, want_energy, split);
    if (gx_orig) k_grad_out<<<nb, bs, 0, st>>>(s, gxc, gx_orig);
    const int64_t chunk = (n + nparts - 1) / nparts;
    k_colsum_partials<<<nparts, CS_THREADS, 0, st>>>(prm, n, ncol, chunk > 0 ? chunk : 1, part);
    k_colsum_final<<<1, CS_THREADS, 0, st>>>(part, nparts, ncol, tot);
}

template <typename K>
static void allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void init_grad_kernels() {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    allow_max_smem(k_force_backward<double>);
    allow_max_smem(k_force_backward<float>);
}

}  // namespace mdgb
