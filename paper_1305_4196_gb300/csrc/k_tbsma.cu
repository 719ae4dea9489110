// k_tbsma.cu - many-body forces of the tight-binding second-moment potential (Cleri and
// Rosato 1993), the potential of all of the paper's benchmarks (Sec. III), in two passes
// over the same cell tasks and full neighbour lists as the pair forces (Sec. II.A).
//
//   E = sum_i [ sum_j phi(r_ij) - sqrt(rho_i) ],  rho_i = sum_j psi(r_ij)
//   phi(r) = A exp(-p (r/r0 - 1)),  psi(r) = xi^2 exp(-2q (r/r0 - 1))
//   F_i = sum_j [ (2p/r0) phi - (q/r0) psi (1/sqrt(rho_i) + 1/sqrt(rho_j)) ] d / r
//
// Pass 1 (density): one thread per atom sums psi over its list; pass 2 (force) needs
// 1/sqrt(rho_j) of every neighbour, so it runs after pass 1 has finished, as its own
// launch, and stages those values into the .w of the tile entries (one species: the
// species bits are not needed there), so one 128-bit load brings a neighbour's
// coordinates and its 1/sqrt(rho).  Each thread
// writes only its own atom in both passes (full lists), so neither needs atomics.
//
// Mixed precision, as the pair kernels: block-frame FP32 coordinates, FP32 pair terms
// (the exponentials as 2^(k dr + l) on the hardware's base-2 exponential), densities and
// forces summed in Q31.32 fixed point (exact, order independent).  A pair whose FP32 r^2
// lies in the band around r_cut^2 is decided by the FP64 definition: its atom is queued
// and finished after the loop by one warp, against the tile still in shared memory.
#include "fixpt.cuh"
#include "tile.cuh"

namespace mdgb {

namespace {

constexpr int TB_THREADS = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// phi and psi at distance r = r2 * rinv (rinv = 1/r)
__device__ __forceinline__ void tb_terms(const TBTable& tb, float r2, float rinv, float& phi, float& psi) {
    const float dr = __fmaf_rn(r2, rinv, -tb.r0);
    phi = ex2_approx(__fmaf_rn(tb.kp, dr, tb.lp));
    psi = ex2_approx(__fmaf_rn(tb.kq, dr, tb.lq));
}

__device__ __forceinline__ float4 tb_disp(const float4& pi, const float4& pj, float& r2) {
    const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
    r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return make_float4(dx, dy, dz, 0.f);
}

// cutoff test of a pair: FP32 outside the band, the FP64 definition inside it
__device__ __forceinline__ bool tb_inside_exact(const DevState& s, const Geometry& g, const TBTable& tb,
                                                const TileMeta& m, int gi, int u, float r2) {
    if (r2 < tb.rc2lo_f) return true;
    if (!(r2 < tb.rc2hi_f)) return false;
    return fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, tile_global_index(m, u), tb.rc2_d);
}

// Stage the tile; returns false (after flagging) when it does not fit.
__device__ __forceinline__ bool tb_stage(const DevState& s, const Geometry& g, const TileOffsets& to, int tile_cap,
                                         TileMeta& m, float4* tile) {
    tile_meta(g, s.cell_start, spatial_block(g, blockIdx.x), m);
    const int T = m.prefix[64];
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return false;
    }
    if (m.prefix[8] == 0) return false;
    tile_stage_f32_cells(m, s.xr, to, tile);
    if (threadIdx.x == 0) tile[T] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);
    return true;
}

__device__ __forceinline__ void tb_store_density(const DevState& s, int gi, long long q, float rep, float* emb,
                                                 bool energy) {
    const float rho = (float)((double)q * 0x1p-32);
    const float inv = rho > 0.f ? rsqrt_approx(rho) : 0.f;
    emb[gi] = inv;
    if (energy) s.pe_atom_f[gi] = rep - rho * inv;  // sum phi - sqrt(rho)
}

}  // namespace

// ---------------------------------------------------------------- pass 1: densities
template <bool EV>
__global__ void __launch_bounds__(TB_THREADS) k_tbsma_density(DevState s, Geometry g, TBTable tb, TileOffsets to,
                                                              int tile_cap, float* __restrict__ emb) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    __shared__ int nqueued;
    float4* tile = reinterpret_cast<float4*>(smem);
    uint16_t* queued = reinterpret_cast<uint16_t*>(tile + tile_cap);
    if (threadIdx.x == 0) nqueued = 0;
    if (!tb_stage(s, g, to, tile_cap, m, tile)) return;
    __syncthreads();
    const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile);
    const int blk0 = m.start[0], nown = m.prefix[8];
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const float4 pi = tile[ui];
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        FixAcc acc{0u, 0u};
        float rep = 0.f;
        bool bad = nch * 8 > FIX_SPLIT_MAX_TERMS;  // longer lists: the warp's 64-bit sums
        for_each_neighbour(reinterpret_cast<const uint4*>(s.nl) + gi, s.np, nch, [&](int u) {
            float r2;
            tb_disp(pi, lds_tile(tile_s, u), r2);
            const bool in = r2 < tb.rc2hi_f;
            bad |= in & !(r2 < tb.rc2lo_f);
            float phi, psi;
            tb_terms(tb, r2, rsqrt_approx(r2), phi, psi);
            fix_add(acc, in ? psi * FS_SCALE : 0.f, 1.0f);  // psi <= xi^2 e^(2q) < 2048: inside the split
            if (EV) rep += in ? phi : 0.f;
        });
        if (bad) {
            queued[atomicAdd(&nqueued, 1)] = (uint16_t)ui;
            continue;
        }
        tb_store_density(s, gi, fix_final(acc, nch * 8), rep, emb, EV);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < nqueued; k += blockDim.x >> 5) {  // exact finish, one warp per atom
        const int ui = queued[k], gi = blk0 + ui;
        const float4 pi = tile[ui];
        const int T = m.prefix[64];
        const int nent = ((s.nl_cnt[gi] + 7) >> 3) * 8;
        long long q = 0;  // exact 64-bit sum (any list length)
        float rep = 0.f;
        for (int e = lane; e < nent; e += 32) {
            const int u = s.nl[((size_t)(e >> 3) * s.np + gi) * 8 + (e & 7)];
            if (u >= T) continue;
            float r2;
            tb_disp(pi, tile[u], r2);
            const bool in = tb_inside_exact(s, g, tb, m, gi, u, r2);
            float phi, psi;
            tb_terms(tb, r2, rsqrt_approx(r2), phi, psi);
            q += fix_term(in ? psi * FS_SCALE : 0.f, 1.0f);
            if (EV) rep += in ? phi : 0.f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            q += __shfl_xor_sync(0xffffffffu, q, o);
            if (EV) rep += __shfl_xor_sync(0xffffffffu, rep, o);
        }
        if (lane == 0) tb_store_density(s, gi, q, rep, emb, EV);
    }
}

// ---------------------------------------------------------------- pass 2: forces
template <bool EV>
__global__ void __launch_bounds__(TB_THREADS) k_tbsma_force(DevState s, Geometry g, TBTable tb, TileOffsets to,
                                                            int tile_cap, const float* __restrict__ emb,
                                                            float fs2_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    __shared__ int nqueued;
    float4* tile = reinterpret_cast<float4*>(smem);  // .w: 1/sqrt(rho) of the atom
    uint16_t* queued = reinterpret_cast<uint16_t*>(tile + tile_cap);
    if (threadIdx.x == 0) nqueued = 0;
    if (!tb_stage(s, g, to, tile_cap, m, tile)) return;
    __syncthreads();  // the coordinates' .w (species) is overwritten below
    tile_stage_w(m, emb, tile);
    __syncthreads();
    const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile);
    const int blk0 = m.start[0], nown = m.prefix[8];
    const int64_t n = s.n;
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const float4 pi = tile[ui];
        const float inv_i = pi.w;
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
        bool bad = nch * 8 > FIX_SPLIT_MAX_TERMS;  // longer lists: the warp's 64-bit sums
        for_each_neighbour(reinterpret_cast<const uint4*>(s.nl) + gi, s.np, nch, [&](int u) {
            float r2;
            const float4 pj = lds_tile(tile_s, u);
            const float4 d = tb_disp(pi, pj, r2);
            const bool in = r2 < tb.rc2hi_f;
            const float rinv = rsqrt_approx(r2);
            float phi, psi;
            tb_terms(tb, r2, rinv, phi, psi);
            const float fr = __fmaf_rn(tb.c_rep, phi, -tb.c_band * psi * (inv_i + pj.w));
            const float fs2 = in ? fr * rinv * FS_SCALE : 0.f;  // (|f| / r) * 2^11
            bad |= (in & !(r2 < tb.rc2lo_f)) | !(fabsf(fs2) < fs2_max);
            fix_add(ax, fs2, d.x);
            fix_add(ay, fs2, d.y);
            fix_add(az, fs2, d.z);
            if (EV) {
                const float gq = fs2 * (1.0f / FS_SCALE);
                w0 += d.x * (gq * d.x);
                w1 += d.y * (gq * d.y);
                w2 += d.z * (gq * d.z);
                w3 += d.x * (gq * d.y);
                w4 += d.x * (gq * d.z);
                w5 += d.y * (gq * d.z);
            }
        });
        if (bad) {
            queued[atomicAdd(&nqueued, 1)] = (uint16_t)ui;
            continue;
        }
        const int nterms = nch * 8;
        s.fq[gi] = fix_final(ax, nterms);
        s.fq[n + gi] = fix_final(ay, nterms);
        s.fq[2 * n + gi] = fix_final(az, nterms);
        if (EV) {  // full lists see every pair twice: each atom keeps half of each pair virial
            s.vir_atom_f[gi] = 0.5f * w0;
            s.vir_atom_f[n + gi] = 0.5f * w1;
            s.vir_atom_f[2 * n + gi] = 0.5f * w2;
            s.vir_atom_f[3 * n + gi] = 0.5f * w3;
            s.vir_atom_f[4 * n + gi] = 0.5f * w4;
            s.vir_atom_f[5 * n + gi] = 0.5f * w5;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < nqueued; k += blockDim.x >> 5) {  // exact finish, one warp per atom
        const int ui = queued[k], gi = blk0 + ui;
        const float4 pi = tile[ui];
        const float inv_i = pi.w;
        const int T = m.prefix[64];
        const int nent = ((s.nl_cnt[gi] + 7) >> 3) * 8;
        long long qx = 0, qy = 0, qz = 0;  // exact 64-bit sums (any list length)
        int nwide = 0;
        float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
        for (int e = lane; e < nent; e += 32) {
            const int u = s.nl[((size_t)(e >> 3) * s.np + gi) * 8 + (e & 7)];
            if (u >= T) continue;
            float r2;
            const float4 pj = tile[u];
            const float4 d = tb_disp(pi, pj, r2);
            const bool in = tb_inside_exact(s, g, tb, m, gi, u, r2);
            const float rinv = rsqrt_approx(r2);
            float phi, psi;
            tb_terms(tb, r2, rinv, phi, psi);
            const float fr = __fmaf_rn(tb.c_rep, phi, -tb.c_band * psi * (inv_i + pj.w));
            const float fs2 = in ? fr * rinv * FS_SCALE : 0.f;
            qx += fix_term_any(fs2, d.x, fs2_max, s.err);
            qy += fix_term_any(fs2, d.y, fs2_max, s.err);
            qz += fix_term_any(fs2, d.z, fs2_max, s.err);
            nwide += fabsf(fs2) < fs2_max ? 0 : 1;
            if (EV) {
                const float gq = fs2 * (1.0f / FS_SCALE);
                w0 += d.x * (gq * d.x);
                w1 += d.y * (gq * d.y);
                w2 += d.z * (gq * d.z);
                w3 += d.x * (gq * d.y);
                w4 += d.x * (gq * d.z);
                w5 += d.y * (gq * d.z);
            }
        }
        nwide = __reduce_add_sync(0xffffffffu, (unsigned)nwide);
        if (lane == 0) fix_wide_count_ok(nwide, s.err);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            qx += __shfl_xor_sync(0xffffffffu, qx, o);
            qy += __shfl_xor_sync(0xffffffffu, qy, o);
            qz += __shfl_xor_sync(0xffffffffu, qz, o);
            if (EV) {
                w0 += __shfl_xor_sync(0xffffffffu, w0, o);
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
                w2 += __shfl_xor_sync(0xffffffffu, w2, o);
                w3 += __shfl_xor_sync(0xffffffffu, w3, o);
                w4 += __shfl_xor_sync(0xffffffffu, w4, o);
                w5 += __shfl_xor_sync(0xffffffffu, w5, o);
            }
        }
        if (lane == 0) {
            s.fq[gi] = qx;
            s.fq[n + gi] = qy;
            s.fq[2 * n + gi] = qz;
            if (EV) {
                s.vir_atom_f[gi] = 0.5f * w0;
                s.vir_atom_f[n + gi] = 0.5f * w1;
                s.vir_atom_f[2 * n + gi] = 0.5f * w2;
                s.vir_atom_f[3 * n + gi] = 0.5f * w3;
                s.vir_atom_f[4 * n + gi] = 0.5f * w4;
                s.vir_atom_f[5 * n + gi] = 0.5f * w5;
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
size_t tbsma_smem_bytes(int tile_cap) {
    return (size_t)tile_cap * sizeof(float4) + (((size_t)tile_cap * sizeof(uint16_t) + 15) & ~(size_t)15);
}

template <typename K>
static void tb_allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void init_tbsma_kernels() {
    tb_allow_max_smem(k_tbsma_density<false>);
    tb_allow_max_smem(k_tbsma_density<true>);
    tb_allow_max_smem(k_tbsma_force<false>);
    tb_allow_max_smem(k_tbsma_force<true>);
}

void launch_tbsma(const DevState& s, const Geometry& g, const TBTable& tb, const TileOffsets& to, int tile_cap,
                  float* emb, int with_energy, cudaStream_t st) {
    if (s.n == 0) return;
    const size_t smem = tbsma_smem_bytes(tile_cap);
    // |fs2 * d| < 2^22 (the exact range of the two-part split) holds when |fs2| < 2^22 / r_cut
    const float fs2_max = (float)(4194304.0 / std::sqrt(tb.rc2_d) * 0.999);
    if (with_energy) {
        k_tbsma_density<true><<<g.nblock, TB_THREADS, smem, st>>>(s, g, tb, to, tile_cap, emb);
        k_tbsma_force<true><<<g.nblock, TB_THREADS, smem, st>>>(s, g, tb, to, tile_cap, emb, fs2_max);
    } else {
        k_tbsma_density<false><<<g.nblock, TB_THREADS, smem, st>>>(s, g, tb, to, tile_cap, emb);
        k_tbsma_force<false><<<g.nblock, TB_THREADS, smem, st>>>(s, g, tb, to, tile_cap, emb, fs2_max);
    }
}

}  // namespace mdgb
