// Device helpers of the o2pic kernels: Philox streams, the single-precision
// transforms used by the collision kinematics, rate-table lookup, CIC cell
// location, block scans and the decoupled look-back.
//
// All floating-point work here is written with explicit fmaf() where a fused
// multiply-add is intended; the library is compiled with --fmad=false, so no
// other contraction happens and every operation rounds as written.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace o2 {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds; multipliers
// 0xD2511F53, 0xCD9E8D57; key bumped by 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Block 0 of the streams of one step and tag for many particles: counter
// (step_lo, tag, 0, step_hi) under key (id, seed).  Round 1 and half of round 2
// do not depend on the id (the counter's third word is 0, and the key's second
// word is the seed), so they are computed once per step (philox_pre) and only
// the rest per particle (philox_id); the result is Philox4x32-10 bit for bit.
struct PhiloxPre {
    uint32_t tag, w1, hi2, lo2, seed;
};
__device__ __forceinline__ PhiloxPre philox_pre(uint32_t step_lo, uint32_t tag, uint32_t step_hi, uint32_t seed) {
    // round 1 with key (id, seed): c1 = (tag ^ id, 0, hi(M0 c0) ^ step_hi ^ seed, lo(M0 c0))
    const uint32_t lo0 = 0xD2511F53u * step_lo;
    const uint32_t hi0 = __umulhi(0xD2511F53u, step_lo);
    const uint32_t z1 = hi0 ^ step_hi ^ seed;
    PhiloxPre p;
    p.tag = tag;
    p.w1 = lo0;
    // round 2: the product of the id-free word z1
    p.hi2 = __umulhi(0xCD9E8D57u, z1);
    p.lo2 = 0xCD9E8D57u * z1;
    p.seed = seed;
    return p;
}
__device__ __forceinline__ uint4 philox_id(const PhiloxPre& p, uint32_t id) {
    const uint32_t x1 = p.tag ^ id;
    uint32_t kx = id + 0x9E3779B9u, ky = p.seed + 0xBB67AE85u;
    const uint32_t lo0 = 0xD2511F53u * x1;
    const uint32_t hi0 = __umulhi(0xD2511F53u, x1);
    uint4 c = make_uint4(p.hi2 ^ kx, p.lo2, hi0 ^ p.w1 ^ ky, lo0);   // after round 2
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        kx += 0x9E3779B9u; ky += 0xBB67AE85u;
        const uint32_t l0 = 0xD2511F53u * c.x;
        const uint32_t h0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t l1 = 0xCD9E8D57u * c.z;
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(h1 ^ c.y ^ kx, l1, h0 ^ c.w ^ ky, l0);
    }
    return c;
}

// Word stream of (key0, seed) at (step, tag): block b = Philox(ctr = (step_lo,
// tag, b, step_hi)); words are consumed in order 4b .. 4b+3.
struct Stream {
    uint4 buf;
    uint32_t key0, seed, step_lo, step_hi, tag, block;
    int pos;
    __device__ __forceinline__ void init(uint32_t k0, uint32_t sd, unsigned long long step, uint32_t tg) {
        key0 = k0; seed = sd; step_lo = (uint32_t)step; step_hi = (uint32_t)(step >> 32); tag = tg; block = 0;
        buf = philox4x32_10(make_uint4(step_lo, tag, 0u, step_hi), make_uint2(key0, seed));
        pos = 0;
    }
    // resume after the first two words of block 0 (given)
    __device__ __forceinline__ void resume(uint32_t k0, uint32_t sd, unsigned long long step, uint32_t tg,
                                           uint4 block0, int p) {
        key0 = k0; seed = sd; step_lo = (uint32_t)step; step_hi = (uint32_t)(step >> 32); tag = tg; block = 0;
        buf = block0; pos = p;
    }
    __device__ __forceinline__ uint32_t next() {
        if (pos == 4) {
            ++block;
            buf = philox4x32_10(make_uint4(step_lo, tag, block, step_hi), make_uint2(key0, seed));
            pos = 0;
        }
        const uint32_t w = (pos == 0) ? buf.x : (pos == 1) ? buf.y : (pos == 2) ? buf.z : buf.w;
        ++pos;
        return w;
    }
};

// u32 -> uniform on [0, 1): 24 random bits, exact.
__device__ __forceinline__ float uniform(uint32_t w) {
    return __uint2float_rn(w >> 8) * 5.9604644775390625e-08f;
}

// Natural log in single precision from the atanh series (Abramowitz & Stegun
// 4.1.27): x = 2^e m, m in [sqrt(1/2), sqrt(2)), t = (m-1)/(m+1),
// ln x = e ln2 + 2t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9).  For normal x > 0.
__device__ __forceinline__ float ln_series(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);   // [1, 2)
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    const float t = (m - 1.0f) / (m + 1.0f);
    const float t2 = t * t;
    float p = fmaf(t2, 0.111111111f, 0.142857143f);
    p = fmaf(t2, p, 0.2f);
    p = fmaf(t2, p, 0.333333333f);
    p = fmaf(t2, p, 1.0f);
    const float lnm = (2.0f * t) * p;
    return fmaf((float)e, 0.693147182f, lnm);
}

// Free flight (the null-collision method's candidate times on the time grid
// of a species' pushes): the number K of pushes before the next candidate is
// Geometric(P_max), P(K >= k) = (1 - P_max)^k, drawn by inversion from one
// word: u = ((w >> 8) + 1/2) 2^-24, K = floor(ln(u) / ln(1 - P_max)), capped.
__device__ __forceinline__ uint32_t flight_gap(uint32_t w, float inv_lnq, float kcap) {
    const float u = (__uint2float_rn(w >> 8) + 0.5f) * 5.9604644775390625e-08f;
    const float k = floorf(ln_series(u) * inv_lnq);
    return (k < kcap) ? (uint32_t)k : (uint32_t)kcap;
}

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
    return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// Marsaglia (1972): uniform point (a, b) of the unit disk -> unit vector
// (2a sqrt(1-s), 2b sqrt(1-s), 1-2s).  Capped rejection loop.
__device__ __forceinline__ void isotropic(Stream& st, float& nx, float& ny, float& nz, unsigned& warn) {
    for (int t = 0; t < MAX_TRIES; ++t) {
        const float a = 2.0f * uniform(st.next()) - 1.0f;
        const float b = 2.0f * uniform(st.next()) - 1.0f;
        const float s = fmaf(a, a, b * b);
        if (s < 1.0f) {
            const float h = 2.0f * sqrtf(1.0f - s);
            nx = a * h; ny = b * h; nz = 1.0f - 2.0f * s;
            return;
        }
    }
    ++warn; nx = 0.0f; ny = 0.0f; nz = 1.0f;
}

// Marsaglia-Bray polar method: two independent standard normals.
__device__ __forceinline__ void normal_pair(Stream& st, float& z0, float& z1, unsigned& warn) {
    for (int t = 0; t < MAX_TRIES; ++t) {
        const float a = 2.0f * uniform(st.next()) - 1.0f;
        const float b = 2.0f * uniform(st.next()) - 1.0f;
        const float s = fmaf(a, a, b * b);
        if (s > 0.0f && s < 1.0f) {
            const float f = sqrtf((-2.0f * ln_series(s)) / s);
            z0 = a * f; z1 = b * f;
            return;
        }
    }
    ++warn; z0 = 0.0f; z1 = 0.0f;
}

__device__ __forceinline__ void maxwellian(Stream& st, float sig, float& vx, float& vy, float& vz, unsigned& warn) {
    float z0, z1, z2, z3;
    normal_pair(st, z0, z1, warn);
    normal_pair(st, z2, z3, warn);
    vx = sig * z0; vy = sig * z1; vz = sig * z2;
}

// ------------------------------------------------------------ rate tables
// Grid position of E: index i and weight w with E = E_i + w (E_{i+1} - E_i),
// read off the float's exponent and top mantissa bits (exact).
__device__ __forceinline__ void grid_locate(float E, int& i, float& w, bool& above) {
    above = false;
    if (!(E >= GRID_EMIN)) { i = 0; w = 0.0f; return; }
    if (E >= GRID_EMAX) { i = NGRID - 1; w = 0.0f; above = true; return; }
    const uint32_t b = __float_as_uint(E);
    i = (int)((b >> (23 - GRID_SUB_BITS)) - GRID_BASE);
    w = __uint2float_rn(b & ((1u << (23 - GRID_SUB_BITS)) - 1u)) * (1.0f / (float)(1u << (23 - GRID_SUB_BITS)));
}

__device__ __forceinline__ float grid_interp(const float* T, int stride, int k, int i, float w) {
    if (i >= NGRID - 1) return T[(NGRID - 1) * stride + k];
    const float a = T[i * stride + k], b = T[(i + 1) * stride + k];
    return fmaf(w, b - a, a);
}

// CIC: cell j and fraction in [0, 1] of position x (x in [0, L)).
__device__ __forceinline__ void cell_of(float x, float inv_dx, int Nc, int& j, float& frac) {
    const float s = x * inv_dx;
    j = (int)s;
    if (j > Nc - 1) j = Nc - 1;
    frac = s - (float)j;
}

__device__ __forceinline__ uint32_t cic_r(float frac) {
    return (uint32_t)(frac * 65536.0f);
}

__device__ __forceinline__ bool is_dead(float x) { return x != x; }

__device__ __forceinline__ float dead_marker() { return __uint_as_float(0x7FC00000u); }

// ------------------------------------------------------------------- scans
// Block-wide exclusive scan of one unsigned per thread (BLOCK threads);
// returns the exclusive prefix, *total gets the sum.  `ws` = 32 words of smem.
template <int NT>
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* ws, unsigned* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned t = (lane < NT / 32) ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const unsigned warp_excl = (warp == 0) ? 0u : ws[warp - 1];
    *total = ws[NT / 32 - 1];
    __syncthreads();
    return warp_excl + x - v;
}

// -------------------------------------------- programmatic dependent launch
// The step kernels are launched with programmatic stream serialization: a
// kernel may be scheduled while its predecessor in the stream still runs.
// pdl_wait() returns once the predecessor has completed and its writes are
// visible (immediately for a normal launch), so every such kernel calls it
// before it reads anything a predecessor wrote.  pdl_trigger() lets the
// successor be scheduled once every block of this grid has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Copy of one discharge's parameters into shared memory (batched launches).
__device__ __forceinline__ void load_params(Params& dst, const Params* src) {
    static_assert(sizeof(Params) % 8 == 0, "Params copied as 64-bit words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (unsigned i = threadIdx.x; i < sizeof(Params) / 8; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// ------------------------------------------------------- decoupled look-back
// Per tile: a flag word = (epoch << 2) | state (1 = aggregate published,
// 2 = inclusive prefix published) and two value words (val[2t] = aggregate,
// val[2t+1] = inclusive prefix), each holding two 32-bit counts.  A value is
// stored before its flag (release) and read after the flag (acquire); the
// aggregate word is never rewritten, so a reader that saw state 1 reads the
// aggregate even if the tile has meanwhile published its prefix.
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long pack2(unsigned a, unsigned b) {
    return (unsigned long long)a | ((unsigned long long)b << 32);
}
__device__ __forceinline__ unsigned long long add2(unsigned long long x, unsigned long long y) {
    return pack2((unsigned)x + (unsigned)y, (unsigned)(x >> 32) + (unsigned)(y >> 32));
}

// Called by one thread.  Publishes the tile's aggregate, walks back to the
// nearest inclusive prefix, publishes its own inclusive prefix and returns
// the exclusive prefix.  Tiles are claimed in increasing order by running
// blocks, so every predecessor is being processed; the wait is still bounded:
// on giving up the error flag is set, *ok = false and the caller skips its
// writes.
constexpr unsigned LOOKBACK_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned long long lookback(unsigned long long* flag, unsigned long long* val,
                                                       unsigned tile, unsigned long long agg,
                                                       unsigned long long epoch, unsigned long long* err,
                                                       bool* ok) {
    *ok = true;
    if (tile == 0) {
        st_relaxed(&val[1], agg);
        st_release(&flag[0], (epoch << 2) | 2ull);
        return 0ull;
    }
    st_relaxed(&val[2 * tile], agg);
    st_release(&flag[tile], (epoch << 2) | 1ull);
    unsigned long long excl = 0ull;
    unsigned spins = 0;
    int j = (int)tile - 1;
    while (j >= 0) {
        const unsigned long long f = ld_acquire(&flag[j]);
        if ((f >> 2) != epoch) {
            if (++spins > LOOKBACK_SPIN_LIMIT) {
                atomicOr(err, ERR_TIMEOUT);
                *ok = false;
                return 0ull;
            }
            if (spins > 64) __nanosleep(64);
            continue;
        }
        if ((f & 3ull) == 2ull) {
            excl = add2(excl, ld_relaxed(&val[2 * j + 1]));
            break;
        }
        excl = add2(excl, ld_relaxed(&val[2 * j]));
        --j;
    }
    st_relaxed(&val[2 * tile + 1], add2(excl, agg));
    st_release(&flag[tile], (epoch << 2) | 2ull);
    return excl;
}

}  // namespace o2
