// fixpt.cuh - Q31.32 fixed-point force sums and neighbour-list traversal shared by the
// mixed-precision force kernels.
//
// Every pair force component q = rint(f * 2^32) is added through an exact split into a
// high part (multiples of 2^-11, rounded by adding a "magic" 1.5 * 2^23 in an FMA) and the
// exact remainder (units of 2^-32), each summed in a 32-bit integer.  Integer sums do not
// depend on order, so a force is the same whatever order its pairs are visited in.
#pragma once

#include "mdgb_internal.cuh"

namespace mdgb {

constexpr float MAGIC = 12582912.0f;   // 1.5 * 2^23: adding it rounds |a| < 2^22 to an integer
constexpr float TWO21 = 2097152.0f;    // 2^21
constexpr float FS_SCALE = 2048.0f;    // 2^11: pair force scaled so that rint() yields multiples of 2^-11

// Exact split of a * 2^21 (a = fs2 * d computed exactly inside the FMA) into
// two integer parts: hi counts units of 2^-11, lo units of 2^-32 (both offset
// by the bit pattern of MAGIC, which the caller removes once per term).
struct FixAcc {
    unsigned hi, lo;  // wrap-around sums; the true sums fit in 32 bits
};

__device__ __forceinline__ void fix_add(FixAcc& acc, float fs2, float d) {
    float t1 = __fmaf_rn(fs2, d, MAGIC);
    float h = __fsub_rn(t1, MAGIC);
    float r = __fmaf_rn(fs2, d, -h);
    float t2 = __fmaf_rn(r, TWO21, MAGIC);
    acc.hi += __float_as_uint(t1);
    acc.lo += __float_as_uint(t2);
}

__device__ __forceinline__ void fix_sub(FixAcc& acc, float fs2, float d) {
    // contribution of -d: exact negation of fix_add's terms
    float t1 = __fmaf_rn(fs2, -d, MAGIC);
    float h = __fsub_rn(t1, MAGIC);
    float r = __fmaf_rn(fs2, -d, -h);
    float t2 = __fmaf_rn(r, TWO21, MAGIC);
    acc.hi += __float_as_uint(t1);
    acc.lo += __float_as_uint(t2);
}

// The same term as one 64-bit integer rint(fs2 * d * 2^21) (units of 2^-32): the two-part
// split of fix_add recombined, so a sum of these equals fix_final of the fix_add sums
// whenever those do not wrap.  Valid for |fs2 * d| < 2^22.
__device__ __forceinline__ long long fix_term(float fs2, float d) {
    const float t1 = __fmaf_rn(fs2, d, MAGIC);
    const float h = __fsub_rn(t1, MAGIC);
    const float r = __fmaf_rn(fs2, d, -h);
    const float t2 = __fmaf_rn(r, TWO21, MAGIC);
    return (long long)(int)(__float_as_uint(t1) - __float_as_uint(MAGIC)) * 2097152LL +
           (long long)(int)(__float_as_uint(t2) - __float_as_uint(MAGIC));
}

// Terms beyond the split (|fs2 * d| >= 2^22, a pair force component of 2048 eps/sigma or
// more): rint(fs2 * d * 2^21) in FP64, exact because the product of two floats is.  The
// sums take terms below FIX_WIDE_LIMIT = 2^54 units (a component below 2^22 = 4.2e6
// eps/sigma; Lennard-Jones atoms closer than about 0.42 sigma exceed it); a larger or
// non-finite term flags ERR_NONFINITE and adds nothing.  With at most FIX_WIDE_MAX_TERMS
// such terms per atom (more also flag ERR_NONFINITE) and every other term below 2^43
// units, an atom's 64-bit total cannot wrap.
constexpr double FIX_WIDE_LIMIT = 18014398509481984.0;  // 2^54
constexpr int FIX_WIDE_MAX_TERMS = 255;

static __device__ __noinline__ long long fix_term_wide(float fs2, float d, uint32_t* err) {
    const double a = (double)fs2 * (double)d * 2097152.0;
    if (!(fabs(a) < FIX_WIDE_LIMIT)) {
        atomicOr(err, ERR_NONFINITE);
        return 0;
    }
    return __double2ll_rn(a);
}

// Exact 64-bit sum of one component for the paths that take terms one at a time (the
// exact finish of an atom, the scalar batch pass): normal terms through fix_term, the
// others through fix_term_wide, whose count is checked by fix_wide_count_ok.
__device__ __forceinline__ long long fix_term_any(float fs2, float d, float fs2_max, uint32_t* err) {
    return fabsf(fs2) < fs2_max ? fix_term(fs2, d) : fix_term_wide(fs2, d, err);
}

__device__ __forceinline__ void fix_wide_count_ok(int nwide, uint32_t* err) {
    if (nwide > FIX_WIDE_MAX_TERMS) atomicOr(err, ERR_NONFINITE);
}

// A sum of fix_add terms is exact while its high part stays inside int32: below
// FIX_SPLIT_MAX_TERMS terms (each high part is below 2^22 in magnitude).
constexpr int FIX_SPLIT_MAX_TERMS = 511;

__device__ __forceinline__ long long fix_final(const FixAcc& acc, int nterms) {
    const int hi = (int)(acc.hi - (unsigned)nterms * __float_as_uint(MAGIC));
    const int lo = (int)(acc.lo - (unsigned)nterms * __float_as_uint(MAGIC));
    return (long long)hi * 2097152LL + (long long)lo;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Chunks 0, 1, ... nch-1 of one list, chunk c at lp[c * stride] (stride in uint4 units),
// two entries per call of body; the next chunk is loaded while this one is used.
template <typename Body>
__device__ __forceinline__ void for_each_neighbour_pair(const uint4* __restrict__ lp, size_t stride, int nch,
                                                        Body&& body) {
    uint4 cur = make_uint4(0u, 0u, 0u, 0u);
    if (nch > 0) cur = __ldcs(lp);
    for (int c = 0; c < nch; ++c) {
        uint4 nxt = cur;
        if (c + 1 < nch) nxt = __ldcs(lp + (size_t)(c + 1) * stride);
        body((int)(cur.x & 0xffffu), (int)(cur.x >> 16));
        body((int)(cur.y & 0xffffu), (int)(cur.y >> 16));
        body((int)(cur.z & 0xffffu), (int)(cur.z >> 16));
        body((int)(cur.w & 0xffffu), (int)(cur.w >> 16));
        cur = nxt;
    }
}

template <typename Body>
__device__ __forceinline__ void for_each_neighbour(const uint4* __restrict__ lp, size_t stride, int nch,
                                                   Body&& body) {
    for_each_neighbour_pair(lp, stride, nch, [&](int u0, int u1) {
        body(u0);
        body(u1);
    });
}

// One tile entry with a single 128-bit shared-memory load (base = shared address of the tile).
__device__ __forceinline__ float4 lds_tile(unsigned base, int u) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(base + ((unsigned)u << 4)));
    return v;
}

// Neighbour lists come in chunks of 8 tile indices (one 16-byte load per chunk,
// chunk c of atom i at uint4 index c * np + i); the last chunk is padded with the
// tile's dummy slot T, which holds a point far outside every cutoff.
#define MDGB_FOR_EACH_NEIGHBOUR(ROW0, NP, NCH, ...)                                         \
    {                                                                                        \
        const uint4* lp_ = (ROW0);                                                           \
        uint4 cur_ = make_uint4(0u, 0u, 0u, 0u);                                             \
        if ((NCH) > 0) cur_ = __ldcs(lp_);                                                   \
        for (int c_ = 0; c_ < (NCH); ++c_) {                                                 \
            uint4 nxt_ = cur_;                                                               \
            if (c_ + 1 < (NCH)) nxt_ = __ldcs(lp_ + (size_t)(c_ + 1) * (NP));                \
            const unsigned w_[4] = {cur_.x, cur_.y, cur_.z, cur_.w};                         \
            _Pragma("unroll") for (int e_ = 0; e_ < 8; ++e_) {                               \
                const int u = (int)((w_[e_ >> 1] >> ((e_ & 1) * 16)) & 0xffffu);             \
                __VA_ARGS__                                                                  \
            }                                                                                \
            cur_ = nxt_;                                                                     \
        }                                                                                    \
    }

// ---------------------------------------------------------------- packed FP32x2 helpers
// sm_100-family packed single-precision arithmetic: two IEEE FP32 operations per
// instruction, each rounded exactly as its scalar counterpart.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Two pairs' fixed-point terms of one component, packed: the same operations as fix_add.
__device__ __forceinline__ void fix_add2(FixAcc& acc, f2_t fs2, f2_t d, f2_t magic2, f2_t two21) {
    const f2_t t1 = f2_fma(fs2, d, magic2);
    const f2_t nh = f2_sub(magic2, t1);  // -h, exact
    const f2_t r = f2_fma(fs2, d, nh);
    const f2_t t2 = f2_fma(r, two21, magic2);
    float t1a, t1b, t2a, t2b;
    f2_unpack(t1, t1a, t1b);
    f2_unpack(t2, t2a, t2b);
    acc.hi += __float_as_uint(t1a) + __float_as_uint(t1b);
    acc.lo += __float_as_uint(t2a) + __float_as_uint(t2b);
}

}  // namespace mdgb
