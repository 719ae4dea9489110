// k_force_fp64.cu - Lennard-Jones forces in FP64 throughout, by cell tasks (Sec. II.A).
//
// The same task structure as the mixed-precision kernels (k_force.cu): one CTA per
// 2x2x2-cell block with the block's 4x4x4-cell tile staged in shared memory, here as FP64
// coordinates relative to the block.
//  * Full lists: one thread per atom i, accumulating only F_i (no particle is written by
//    two workers, Sec. II.A).
//  * Half lists (Newton's third law, Sec. II.D.3): the reaction -f_ij goes to the tile copy
//    of j in shared memory; one launch per colour class of blocks, whose tiles are disjoint
//    (the barrier-separated waves of Sec. II.B).
//
// On GB300 the FP64 pipe bounds these kernels (the list and coordinates stream through
// with DRAM nearly idle), so the pair arithmetic is kept to few FP64 operations: one
// reciprocal of r^2 per pair serves both (sigma/r)^2 and f/r.
#include "fixpt.cuh"
#include "tile.cuh"

#include <algorithm>

namespace mdgb {

constexpr int F_THREADS = 256;
static int g_sm_count = 0;  // SMs of the device, read at initialisation (never during a stream capture)

// 1/x to within about an ulp: the hardware's approximate reciprocal, refined by two
// Newton-Raphson steps y <- y + y (1 - x y), each of which doubles the correct bits (a
// seed good to 2^-14 or better reaches full precision).  For x = 0 the result is not
// finite, and the force kernels flag the non-finite force.
__device__ __forceinline__ double rcp_nr(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double e = fma(-x, y, 1.0);
        y = fma(y, e, y);
    }
    return y;
}

// ---------------------------------------------------------------- full list
template <bool EV>
__global__ void __launch_bounds__(F_THREADS) k_force_fp64_full(DevState s, Geometry g, PairTable pt, int tile_cap,
                                                               int split) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    double* tx = reinterpret_cast<double*>(smem);
    double* ty = tx + tile_cap;
    double* tz = ty + tile_cap;
    int* tsp = reinterpret_cast<int*>(tz + tile_cap);
    // split CTAs share one block (small systems): each stages the tile and takes every
    // split-th group of F_THREADS own atoms
    const int b = spatial_block(g, blockIdx.x / split), part = blockIdx.x % split;
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    tile_stage_f64(s, g, m, b, tx, ty, tz, tsp);
    __syncthreads();
    const int blk0 = m.start[0];
    const int nown = m.prefix[8];
    const int64_t n = s.n;
    const int np = s.np;
    for (int ui = part * blockDim.x + threadIdx.x; ui < nown; ui += split * blockDim.x) {
        const int gi = blk0 + ui;
        const double xi = tx[ui], yi = ty[ui], zi = tz[ui];
        const int si = tsp[ui];
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        double fx = 0, fy = 0, fz = 0, pe = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
        MDGB_FOR_EACH_NEIGHBOUR(reinterpret_cast<const uint4*>(s.nl) + gi, np, nch, {
            const double dx = xi - tx[u], dy = yi - ty[u], dz = zi - tz[u];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const int t = si * pt.nsp + tsp[u];
            if (r2 < pt.rc2_d[t]) {
                const double inv = rcp_nr(r2);
                const double sr2 = pt.sig2_d[t] * inv;
                const double s6 = sr2 * sr2 * sr2;
                const double e = pt.eps_d[t];
                const double fr = 24.0 * e * (2.0 * s6 * s6 - s6) * inv;
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                if (EV) {
                    pe += 4.0 * e * (s6 * s6 - s6);
                    w0 += dx * (fr * dx);
                    w1 += dy * (fr * dy);
                    w2 += dz * (fr * dz);
                    w3 += dx * (fr * dy);
                    w4 += dx * (fr * dz);
                    w5 += dy * (fr * dz);
                }
            }
        })
        if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(s.err, ERR_NONFINITE);
        s.f[gi] = fx;
        s.f[n + gi] = fy;
        s.f[2 * n + gi] = fz;
        if (EV) {
            s.pe_atom_d[gi] = 0.5 * pe;
            s.vir_atom_d[gi] = 0.5 * w0;
            s.vir_atom_d[n + gi] = 0.5 * w1;
            s.vir_atom_d[2 * n + gi] = 0.5 * w2;
            s.vir_atom_d[3 * n + gi] = 0.5 * w3;
            s.vir_atom_d[4 * n + gi] = 0.5 * w4;
            s.vir_atom_d[5 * n + gi] = 0.5 * w5;
        }
    }
}

// FP64 half list, one colour: reactions through FP64 shared-memory accumulators.
template <bool EV>
__global__ void __launch_bounds__(F_THREADS) k_force_fp64_half(DevState s, Geometry g, PairTable pt, int tile_cap,
                                                               int block0) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    double* tx = reinterpret_cast<double*>(smem);
    double* ty = tx + tile_cap;
    double* tz = ty + tile_cap;
    double* acc = tz + tile_cap;  // 3 x tile_cap
    int* tsp = reinterpret_cast<int*>(acc + 3 * tile_cap);
    const int b = block0 + blockIdx.x;
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    tile_stage_f64(s, g, m, b, tx, ty, tz, tsp);
    for (int u = threadIdx.x; u <= T; u += blockDim.x) {
        acc[u] = 0;
        acc[tile_cap + u] = 0;
        acc[2 * tile_cap + u] = 0;
    }
    __syncthreads();
    const int blk0 = m.start[0];
    const int nown = m.prefix[8];
    const int64_t n = s.n;
    const int np = s.np;
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const double xi = tx[ui], yi = ty[ui], zi = tz[ui];
        const int si = tsp[ui];
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        double fx = 0, fy = 0, fz = 0, pe = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
        MDGB_FOR_EACH_NEIGHBOUR(reinterpret_cast<const uint4*>(s.nl) + gi, np, nch, {
            const double dx = xi - tx[u], dy = yi - ty[u], dz = zi - tz[u];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const int t = si * pt.nsp + tsp[u];
            if (r2 < pt.rc2_d[t]) {
                const double inv = rcp_nr(r2);
                const double sr2 = pt.sig2_d[t] * inv;
                const double s6 = sr2 * sr2 * sr2;
                const double e = pt.eps_d[t];
                const double fr = 24.0 * e * (2.0 * s6 * s6 - s6) * inv;
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                atomicAdd(&acc[u], -fr * dx);
                atomicAdd(&acc[tile_cap + u], -fr * dy);
                atomicAdd(&acc[2 * tile_cap + u], -fr * dz);
                if (EV) {
                    pe += 4.0 * e * (s6 * s6 - s6);
                    w0 += dx * (fr * dx);
                    w1 += dy * (fr * dy);
                    w2 += dz * (fr * dz);
                    w3 += dx * (fr * dy);
                    w4 += dx * (fr * dz);
                    w5 += dy * (fr * dz);
                }
            }
        })
        // a non-finite pair force leaves its mark on the i-side sum (a pair at r = 0 gives inf * 0)
        if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(s.err, ERR_NONFINITE);
        atomicAdd(&acc[ui], fx);
        atomicAdd(&acc[tile_cap + ui], fy);
        atomicAdd(&acc[2 * tile_cap + ui], fz);
        if (EV) {
            s.pe_atom_d[gi] = pe;
            s.vir_atom_d[gi] = w0;
            s.vir_atom_d[n + gi] = w1;
            s.vir_atom_d[2 * n + gi] = w2;
            s.vir_atom_d[3 * n + gi] = w3;
            s.vir_atom_d[4 * n + gi] = w4;
            s.vir_atom_d[5 * n + gi] = w5;
        }
    }
    __syncthreads();
    for (int u = threadIdx.x; u < T; u += blockDim.x) {
        const int slot = tile_slot_of(m, u);
        const int gj = m.start[slot] + (u - m.prefix[slot]);
        s.f[gj] += acc[u];
        s.f[n + gj] += acc[tile_cap + u];
        s.f[2 * n + gj] += acc[2 * tile_cap + u];
    }
}

// ---------------------------------------------------------------- launchers
void launch_forces_fp64(const DevState& s, const Geometry& g, const PairTable& pt, int tile_cap, int half,
                        int with_energy, cudaStream_t st) {
    if (s.n == 0) return;
    const size_t smem = force_smem_bytes(0, half, with_energy, tile_cap);
    if (!half) {
        // CTAs per block: about one own atom per thread while the grid is below two CTAs per SM
        const int sms = g_sm_count > 0 ? g_sm_count : 152;
        const int64_t per_block = (s.n + g.nblock - 1) / g.nblock;
        int split = (int)std::min<int64_t>((per_block + F_THREADS - 1) / F_THREADS, (2 * sms + g.nblock - 1) / g.nblock);
        split = std::max(1, std::min(split, 8));
        const unsigned grid = (unsigned)g.nblock * (unsigned)split;
        if (with_energy) {
            k_force_fp64_full<true><<<grid, F_THREADS, smem, st>>>(s, g, pt, tile_cap, split);
        } else {
            k_force_fp64_full<false><<<grid, F_THREADS, smem, st>>>(s, g, pt, tile_cap, split);
        }
        return;
    }
    cudaMemsetAsync(s.f, 0, sizeof(double) * 3 * (size_t)s.n, st);
    const int per = g.nblock / 8;
    for (int col = 0; col < 8; ++col) {
        if (with_energy) {
            k_force_fp64_half<true><<<per, F_THREADS, smem, st>>>(s, g, pt, tile_cap, col * per);
        } else {
            k_force_fp64_half<false><<<per, F_THREADS, smem, st>>>(s, g, pt, tile_cap, col * per);
        }
    }
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

void init_force_fp64_kernels() {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    allow_max_smem(k_force_fp64_full<false>);
    allow_max_smem(k_force_fp64_full<true>);
    allow_max_smem(k_force_fp64_half<false>);
    allow_max_smem(k_force_fp64_half<true>);
}

}  // namespace mdgb
