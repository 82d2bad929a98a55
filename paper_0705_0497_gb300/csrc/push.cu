// Particle kernel of one species for one time step (Sec. 2 of the paper):
// field gather, leapfrog push in x (v_x accelerated, v_y and v_z carried),
// absorbing electrodes, null-collision Monte Carlo against the O2 / O2(a)
// background, births, and the CIC charge deposit of the pushed particles.
//
// Layout and flow (GB300-first):
//   * SoA FP32 arrays x, vx, vy, vz + u32 id, updated IN PLACE: a particle
//     keeps its slot, removed particles are marked (x = NaN) and dropped by a
//     periodic stable compaction, births are appended after the last slot.
//     The common path reads x, vx, tc (12 B) and writes x, vx (8 B); id,
//     vy, vz are read for collision candidates only.
//   * a persistent grid; each warp owns one contiguous, 128-aligned slot range
//     and walks it in rounds of 128 (lane l takes slots l, l+32, l+64, l+96:
//     every load and store is one coalesced 128-byte line per array).  No
//     block-wide barrier between the set-up and the final flush.
//   * the gather field and the deposit live in shared memory; the deposit is
//     one 64-bit atomic per particle holding (count, sum of CIC weights) per
//     cell, turned into node charges when the block flushes;
//   * free flights (Sec. 2: "the durations of the free flights ... from
//     elementary kinetic considerations"): each particle carries the step of
//     its next null-collision candidate (tc, read with x and v_x), so the
//     common path draws no random number; candidates are queued per warp in
//     shared memory and handled 32 at a time (all lanes busy): one Philox
//     block (the id-free first round hoisted) draws the next free flight and
//     the rest of the collision;
//   * electrons: a candidate is filtered at once (energy against the total
//     rate, the total-rate column in shared memory), only the real
//     collisions are recorded (32 B each: slot, id, x, v), and the warp runs
//     their kinematics itself once its range is pushed, while other warps
//     are still pushing (no second kernel on electron steps);
//   * ions: candidates are recorded (slot and the rest of the Philox block),
//     a lean filter kernel (target sampled from the gas Maxwellian, energy
//     against the total rate) keeps the real ones, and the kinematics kernel
//     handles those, 32 at a time;
//   * births are ranked with warp ballots and staged at the warp's range;
//     the end-of-step kernel places them in parent order.
#include "common.cuh"

// Launch shape of the particle kernels: minimum resident blocks per SM (caps
// the registers; 4 timed fastest of 2, 3, 4 on the 512-cell, 1.6e7-particle
// workload) and unrolling of the four particles a lane handles per round.
#ifndef O2PIC_PUSH_MIN_BLOCKS
#define O2PIC_PUSH_MIN_BLOCKS 4
#endif
// The electron kernel also runs the kinematics of its real collisions.
#ifndef O2PIC_PUSH_E_MIN_BLOCKS
#define O2PIC_PUSH_E_MIN_BLOCKS 4
#endif
// Ion candidates filtered (gas target, energy against the total rate) and
// their real collisions handled inside the particle kernel, as for the
// electrons (1), or by the separate filter and kinematics kernels (0).  Both
// give the same results; on the 512-cell, 1.6e7-particle discharge at its
// periodic state the separate kernels were faster (48.4 against 49.1 ms per
// RF cycle): the ion filter's Maxwellian target draws weigh on the particle
// kernel's registers.
#ifndef O2PIC_FUSE_IONS
#define O2PIC_FUSE_IONS 0
#endif
// Deposit: one 64-bit shared-memory atomic per particle (0), or lanes of a
// warp that hit the same cell first summed over __match_any_sync peers and
// added by one lane (1).  Integers: both give the same charge.  The
// aggregated form was far slower on the 512-cell discharge (76.7 against
// 46.3 ms per RF cycle): the lanes of a warp rarely share a cell, and the
// match and the shuffles cost more than the atomics they save.
#ifndef O2PIC_DEPOSIT_AGG
#define O2PIC_DEPOSIT_AGG 0
#endif
// The particle kernel that runs the kinematics stages the species' cumulative
// rate table in shared memory when that keeps its resident blocks per SM (1),
// or reads it from global memory through L1 (0).  Both give the same results;
// on the 512-cell, 1.6e7-particle discharge at its periodic state the global
// table was faster (46.3 against 47.5 ms per RF cycle): every block copies
// the electrons' 34 KB table each step, and the kinematics read a few rows.
#ifndef O2PIC_CUM_SMEM
#define O2PIC_CUM_SMEM 0
#endif
#ifndef O2PIC_PUSH_UNROLL
#define O2PIC_PUSH_UNROLL 4
#endif
// Minimum resident blocks per SM of the kinematics kernel (caps its registers
// at 85, no spills; 3 timed fastest of 2, 3, 4 on the same workload).
#ifndef O2PIC_CAND_MIN_BLOCKS
#define O2PIC_CAND_MIN_BLOCKS 3
#endif

namespace o2 {

namespace {

template <int S> struct SpeciesTraits;
template <> struct SpeciesTraits<SP_E> { static constexpr uint32_t tag = TAG_E; };
template <> struct SpeciesTraits<SP_OM> { static constexpr uint32_t tag = TAG_OM; };
template <> struct SpeciesTraits<SP_OP> { static constexpr uint32_t tag = TAG_OP; };

constexpr int WARPS = BLOCK / 32;           // 8
constexpr int ROUND = 128;                  // slots per warp round (4 per lane)
constexpr int PUSH_UNROLL = O2PIC_PUSH_UNROLL;

struct PushShared {
    unsigned long long jsum;     // block's sum of trunc(256 v_x^{n+1/2})
    unsigned absorbed[2];
    unsigned removed;
    unsigned psteps;
    unsigned nonfinite;
    unsigned wtries;
    unsigned events[MAXPROC];    // electrons: real collisions per process
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// One real collision (a candidate its filter kept) through process selection
// and kinematics, exactly in the order of the oracle.  The filter already
// counted the warnings of the part it shares with this function (the ions'
// target sample, the energy above the grid), so they are not counted again.
// Returns the event index, or -1 for a null collision (the selected
// process's threshold above E; the rate test itself repeats the filter's).
// bkind: 0 none, 1 ionization (two births), 2 attachment / detachment (one).
template <int S>
__device__ __forceinline__ int collide(const Params& P, const float* cum, int np, unsigned long long step,
                                       uint32_t id, uint4 w0, float x, float& vx, float& vy, float& vz,
                                       bool& alive, int& bkind, float4& b1, float4& b2,
                                       unsigned& warn_tries, unsigned& warn_emax) {
    alive = true;
    bkind = 0;
    Stream st;
    st.resume(id, P.seed, step, SpeciesTraits<S>::tag, w0, 1);
    const float u1 = uniform(st.next());
    float vtx = 0.0f, vty = 0.0f, vtz = 0.0f;
    float gx = vx, gy = vy, gz = vz;
    if (S != SP_E) {
        unsigned counted_by_filter = 0;
        maxwellian(st, P.sig_gas, vtx, vty, vtz, counted_by_filter);
        gx = vx - vtx; gy = vy - vty; gz = vz - vtz;
    }
    const float E = P.kappa[S] * dot3(gx, gy, gz, gx, gy, gz);
    int i; float w; bool above;
    grid_locate(E, i, w, above);
    (void)warn_emax;
    // null collision unless u1 nu_max falls below the total rate; then the
    // first process whose cumulative rate exceeds it (the last one if
    // rounding leaves none)
    // the cumulative rates are read four processes at a time (loads in
    // flight together); each value is grid_interp(cum, np, kk, i, w)
    const float target = u1 * P.numax[S];
    const bool last = i >= NGRID - 1;
    const float* row = cum + (size_t)(last ? NGRID - 1 : i) * np;
    auto interp = [&](float a, float b) { return last ? a : fmaf(w, b - a, a); };
    const float ta = row[np - 1], tb = last ? 0.0f : row[2 * np - 1];
    float a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a[j] = (j < np - 1) ? row[j] : 0.0f;
        b[j] = (j < np - 1 && !last) ? row[np + j] : 0.0f;
    }
    if (!(target < interp(ta, tb))) return -1;
    int k = np - 1;
    for (int k0 = 0; k0 < np - 1; k0 += 4) {
        if (k0 > 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kk = k0 + j;
                a[j] = (kk < np - 1) ? row[kk] : 0.0f;
                b[j] = (kk < np - 1 && !last) ? row[np + kk] : 0.0f;
            }
        }
        int f = -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = k0 + j;
            if (f < 0 && kk < np - 1 && target < interp(a[j], b[j])) f = kk;
        }
        if (f >= 0) { k = f; break; }
    }
    const float thr = P.thr[S][k];
    if (E < thr) return -1;
    const int kind = P.kind[S][k];
    if (kind == K_ELASTIC) {
        float nx, ny, nz;
        isotropic(st, nx, ny, nz, warn_tries);
        if (S == SP_E) {
            const float v2 = dot3(vx, vy, vz, vx, vy, vz);
            const float vm = sqrtf(v2);
            const float cosx = (vm > 0.0f) ? dot3(nx, ny, nz, vx, vy, vz) / vm : 0.0f;
            const float fac = 1.0f - P.delta_el * (1.0f - cosx);
            const float vn = vm * sqrtf(fac);
            vx = vn * nx; vy = vn * ny; vz = vn * nz;
        } else {
            const float gm = sqrtf(dot3(gx, gy, gz, gx, gy, gz));
            const float cmx = fmaf(P.a_m[S], vx, P.a_M[S] * vtx);
            const float cmy = fmaf(P.a_m[S], vy, P.a_M[S] * vty);
            const float cmz = fmaf(P.a_m[S], vz, P.a_M[S] * vtz);
            const float f = P.a_M[S] * gm;
            vx = fmaf(f, nx, cmx); vy = fmaf(f, ny, cmy); vz = fmaf(f, nz, cmz);
        }
    } else if (kind == K_EXCITE) {
        const float Ep = E - thr;
        float nx, ny, nz;
        isotropic(st, nx, ny, nz, warn_tries);
        const float vn = sqrtf(Ep / P.kappa[S]);
        vx = vn * nx; vy = vn * ny; vz = vn * nz;
    } else if (kind == K_IONIZE) {
        const float Er = E - thr;
        const float u = uniform(st.next());
        const float Es = u * Er;
        const float Epr = Er - Es;
        float n1x, n1y, n1z, n2x, n2y, n2z, vix, viy, viz;
        isotropic(st, n1x, n1y, n1z, warn_tries);
        isotropic(st, n2x, n2y, n2z, warn_tries);
        maxwellian(st, P.sig_birth[SP_OP], vix, viy, viz, warn_tries);
        const float vp = sqrtf(Epr / P.kappa[SP_E]);
        const float vs = sqrtf(Es / P.kappa[SP_E]);
        vx = vp * n1x; vy = vp * n1y; vz = vp * n1z;
        b1 = make_float4(x, vs * n2x, vs * n2y, vs * n2z);
        b2 = make_float4(x, vix, viy, viz);
        bkind = 1;
    } else if (kind == K_ATTACH) {
        float vix, viy, viz;
        maxwellian(st, P.sig_birth[SP_OM], vix, viy, viz, warn_tries);
        b1 = make_float4(x, vix, viy, viz);
        bkind = 2;
        alive = false;
    } else if (kind == K_DETACH) {
        const float Er = E - thr;
        float nx, ny, nz;
        isotropic(st, nx, ny, nz, warn_tries);
        const float vn = sqrtf(Er / P.kappa[SP_E]);
        b1 = make_float4(x, vn * nx, vn * ny, vn * nz);
        bkind = 2;
        alive = false;
    } else if (kind == K_CX) {
        vx = vtx; vy = vty; vz = vtz;
    }
    return k;
}

__device__ __forceinline__ void deposit_add(unsigned* hist, float x, float inv_dx, int Nc) {
    int j; float frac;
    cell_of(x, inv_dx, Nc, j, frac);
    const uint32_t r = cic_r(frac);
    atomicAdd(&hist[j], 65536u - r);
    atomicAdd(&hist[j + 1], r);
}

__device__ __forceinline__ void deposit_sub_global(unsigned long long* Q, float x, float inv_dx, int Nc) {
    int j; float frac;
    cell_of(x, inv_dx, Nc, j, frac);
    const uint32_t r = cic_r(frac);
    atomicAdd(&Q[j], 0ull - (unsigned long long)(65536u - r));
    atomicAdd(&Q[j + 1], 0ull - (unsigned long long)r);
}

// A birth's CIC charge, into the births' accumulator Qb of its species.
__device__ __forceinline__ void deposit_add_global(unsigned long long* Q, float x, float inv_dx, int Nc) {
    int j; float frac;
    cell_of(x, inv_dx, Nc, j, frac);
    const uint32_t r = cic_r(frac);
    atomicAdd(&Q[j], (unsigned long long)(65536u - r));
    if (r) atomicAdd(&Q[j + 1], (unsigned long long)r);
}

__device__ __forceinline__ void flush_hist(unsigned* hist, unsigned long long* Q, int Ng) {
    for (int j = threadIdx.x; j < Ng; j += BLOCK) {
        const unsigned v = hist[j];
        if (v) {
            atomicAdd(&Q[j], (unsigned long long)v);
            hist[j] = 0u;
        }
    }
}

// Filter of an electron candidate: is it a real collision?  The same
// arithmetic as the start of collide(): energy of the particle, the total
// rate on the table grid (column `tot` = the last cumulative column) and the
// comparison with u1 nu_max.
__device__ __forceinline__ bool electron_is_real(const Params& P, const float* tot, uint32_t w1, float vx, float vy,
                                                 float vz, unsigned& wemax, unsigned& wnumax) {
    const float u1 = uniform(w1);
    const float E = P.kappa[SP_E] * dot3(vx, vy, vz, vx, vy, vz);
    int i; float w; bool above;
    grid_locate(E, i, w, above);
    if (above) ++wemax;
    const float total = grid_interp(tot, 1, 0, i, w);
    if (total > P.numax[SP_E]) ++wnumax;   // above a capped majorant
    return (u1 * P.numax[SP_E]) < total;
}

// Filter of an ion candidate: the target sampled from the gas Maxwellian
// (words 2, 3 of block 0 and the blocks after), the relative energy, and the
// total rate on the table grid against u1 nu_max (word 1): the same
// arithmetic as the start of collide().
template <int S>
__device__ __forceinline__ bool ion_is_real(const Params& P, const float* tot, unsigned long long step, uint32_t id,
                                            uint4 w, float vx, float vy, float vz, unsigned& wtries,
                                            unsigned& wemax, unsigned& wnumax) {
    Stream st;
    st.resume(id, P.seed, step, SpeciesTraits<S>::tag, w, 1);
    const float u1 = uniform(st.next());
    float vtx, vty, vtz;
    maxwellian(st, P.sig_gas, vtx, vty, vtz, wtries);
    const float gx = vx - vtx, gy = vy - vty, gz = vz - vtz;
    const float E = P.kappa[S] * dot3(gx, gy, gz, gx, gy, gz);
    int i; float wt; bool above;
    grid_locate(E, i, wt, above);
    if (above) ++wemax;
    const float total = grid_interp(tot, 1, 0, i, wt);
    if (total > P.numax[S]) ++wnumax;   // above a capped majorant
    return (u1 * P.numax[S]) < total;
}

// Total-rate column (the last cumulative column) of species S into shared memory.
__device__ __forceinline__ void stage_total(const Params& P, int S, float* tot) {
    const int np = P.nproc[S];
    const float* __restrict__ cum = P.cum[S];
    for (int i = threadIdx.x; i < NGRID; i += blockDim.x) tot[i] = np > 0 ? cum[(size_t)i * np + np - 1] : 0.0f;
}

// Real collisions of the list of one particle-kernel warp (records r0 ..
// r0 + n - 1, in slot order), taken SEGW records per pass by the SEGW lanes
// of one segment of the calling warp (seg_mask: its lanes; sl: this lane's
// index in it; lt_mask: the segment's lanes below this one; nmax: the longest
// list among the warp's segments, so that every lane makes the same passes).
// Electron records carry the particle (slot, id, x, v) and block 0 of its
// Philox stream is drawn again; ion records carry the slot, id, v and that
// block (its first word, the candidate draw, is spent), x is read from the
// array.  `cum` is the species' cumulative rate table (global or shared
// memory).  A removed particle's charge comes off the block's histogram when
// `hist` is given (the particle kernel: the particle was deposited there),
// else off the step's deposit in global memory.  Births are ranked with
// ballots within the segment and staged at the particle warp's slot range;
// nb1, nb2 count them.
template <int S, int SEGW>
__device__ __forceinline__ void collide_list(const Params& P, const float* cum, const PhiloxPre& pre,
                                             unsigned long long step,
                                             unsigned r0, unsigned n, unsigned nmax, unsigned sl,
                                             unsigned seg_mask, unsigned lt_mask, unsigned* events,
                                             unsigned long long* hist, unsigned& nb1, unsigned& nb2,
                                             unsigned& nremoved, unsigned& wtries, unsigned& wemax) {
    const int np = P.nproc[S];
    const unsigned cb = P.ctrl->cur[S];
    float* __restrict__ X = P.sp[S].x[cb];
    float* __restrict__ VX = P.sp[S].vx[cb];
    float* __restrict__ VY = P.sp[S].vy[cb];
    float* __restrict__ VZ = P.sp[S].vz[cb];
    const uint4* __restrict__ CAND = P.cand[S];
    const float inv_dx = P.inv_dx;
    const int Nc = P.Nc;
    const bool births = P.births_possible[S] != 0;
    for (unsigned c0 = 0; c0 < nmax; c0 += SEGW) {
        const unsigned ci = c0 + sl;
        const bool has = ci < n;
        uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
        if (has) { a = CAND[2 * (size_t)(r0 + ci)]; b = CAND[2 * (size_t)(r0 + ci) + 1]; }
        const unsigned slot = a.x;
        float x, vx, vy, vz;
        uint4 w0;
        if (S == SP_E) {
            x = __uint_as_float(a.z); vx = __uint_as_float(a.w);
            vy = __uint_as_float(b.x); vz = __uint_as_float(b.y);
            w0 = has ? philox_id(pre, a.y) : make_uint4(0u, 0u, 0u, 0u);
        } else {
            x = has ? X[slot] : 0.0f;
            vx = __uint_as_float(a.z); vy = __uint_as_float(a.w); vz = __uint_as_float(b.x);
            w0 = make_uint4(0u, b.y, b.z, b.w);
        }
        w0.x = a.y;   // word 0 (the candidate draw) is spent: it carries the id
        int bkind = 0;
        float4 b1 = make_float4(0.f, 0.f, 0.f, 0.f), b2 = b1;
        if (has) {
            bool alive;
            const int k = collide<S>(P, cum, np, step, a.y, w0, x, vx, vy, vz, alive, bkind, b1, b2, wtries, wemax);
            if (k >= 0) {
                atomicAdd(&events[k], 1u);
                if (alive) {
                    VX[slot] = vx; VY[slot] = vy; VZ[slot] = vz;
                } else {
                    X[slot] = dead_marker();
                    if (hist) {
                        int j; float f;
                        cell_of(x, inv_dx, Nc, j, f);
                        atomicAdd(&hist[j], 0ull - ((1ull << 40) + (unsigned long long)cic_r(f)));
                    } else {
                        deposit_sub_global(P.Qf[S], x, inv_dx, Nc);
                    }
                    ++nremoved;
                }
            }
        }
        if (births) {
            const unsigned m1 = __ballot_sync(0xffffffffu, bkind == 1) & seg_mask;
            const unsigned m2 = __ballot_sync(0xffffffffu, bkind == 2) & seg_mask;
            // staged for the end-of-step kernel, which places them; their
            // charge goes to Qb now
            if (S == SP_E) {
                if (bkind == 1) {
                    const unsigned r = nb1 + __popc(m1 & lt_mask);
                    P.stage[B_E_FROM_E][r0 + r] = b1;
                    P.stage[B_OP_FROM_E][r0 + r] = b2;
                    deposit_add_global(P.Qb[SP_E], b1.x, inv_dx, Nc);
                    deposit_add_global(P.Qb[SP_OP], b2.x, inv_dx, Nc);
                } else if (bkind == 2) {
                    P.stage[B_OM_FROM_E][r0 + nb2 + __popc(m2 & lt_mask)] = b1;
                    deposit_add_global(P.Qb[SP_OM], b1.x, inv_dx, Nc);
                }
            } else if (S == SP_OM) {
                if (bkind == 2) {
                    P.stage[B_E_FROM_OM][r0 + nb2 + __popc(m2 & lt_mask)] = b1;
                    deposit_add_global(P.Qb[SP_E], b1.x, inv_dx, Nc);
                }
            }
            nb1 += __popc(m1);
            nb2 += __popc(m2);
        }
        __syncwarp();
    }
}

// Candidate queue of one warp of the particle kernel (shared memory): slot,
// x and v_x after the push of up to QN candidates in slot order.
constexpr int QN = 64;
struct PushQueue {
    unsigned slot[WARPS][QN];
    float x[WARPS][QN];
    float vx[WARPS][QN];
};

// Body of the particle kernel for block blk of nblk blocks (the launch's own
// block, or a block a batched launch maps to this discharge).
template <int S>
__device__ __forceinline__ void push_body(const Params& P, unsigned blk, unsigned nblk) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = P.nproc[S];
    PushShared& sh = *reinterpret_cast<PushShared*>(smem);
    float* Es = reinterpret_cast<float*>(smem + align16(sizeof(PushShared)));
    unsigned long long* hist =
        reinterpret_cast<unsigned long long*>(smem + align16(align16(sizeof(PushShared)) + sizeof(float) * P.Ng));
    PushQueue& Q = *reinterpret_cast<PushQueue*>(hist + P.Ng);
    float* Tt = reinterpret_cast<float*>(&Q + 1);        // total-rate column (filter in the kernel)
    float* Ct = Tt + NGRID;                              // cumulative table (if staged)
    constexpr bool fused = (S == SP_E) || (O2PIC_FUSE_IONS != 0);
    const bool cum_staged = fused && P.cum_smem[S] != 0;
    const float* cum = cum_staged ? Ct : P.cum[S];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned* qs = Q.slot[warp];
    float* qx = Q.x[warp];
    float* qv = Q.vx[warp];

    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const uint32_t step_lo = (uint32_t)step;
    const unsigned cb = C->cur[S];
    const unsigned nslots = (unsigned)((C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap);
    float* __restrict__ X = P.sp[S].x[cb];
    float* __restrict__ VX = P.sp[S].vx[cb];
    const float* __restrict__ VY = P.sp[S].vy[cb];
    const float* __restrict__ VZ = P.sp[S].vz[cb];
    const uint32_t* __restrict__ ID = P.sp[S].id[cb];
    uint32_t* __restrict__ TC = P.sp[S].tc[cb];
    uint4* __restrict__ CAND = P.cand[S];
    const float qmdt = P.qmdt[S], dts = P.dt_s[S], inv_dx = P.inv_dx, Lf = P.Lf;
    const float inv_lnq = P.inv_lnq[S], kcap = P.kcap[S];
    const unsigned sub = P.sub[S];
    const int Nc = P.Nc, Ng = P.Ng;
    const PhiloxPre pre = philox_pre(step_lo, SpeciesTraits<S>::tag, (uint32_t)(step >> 32), P.seed);

    // this warp's contiguous slot range, and its first round of x, v_x, tc
    // requested before the block's set-up (their latency overlaps it)
    const unsigned W = nblk * WARPS;
    const unsigned gw = blk * WARPS + warp;
    const unsigned R = warp_range_len(nslots, W);
    const unsigned r0 = (gw * (unsigned long long)R < nslots) ? gw * R : nslots;
    const unsigned r1 = (r0 + R < nslots) ? r0 + R : nslots;
    float xs[4], vxs[4];
    uint32_t tcs[4];
    auto load_round = [&](unsigned g0) {
        const bool full = g0 + ROUND <= r1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned i = g0 + 32u * k + lane;
            const bool inr = full || i < r1;
            xs[k] = inr ? X[i] : dead_marker();
            vxs[k] = inr ? VX[i] : 0.0f;
            tcs[k] = inr ? TC[i] : 0u;
        }
    };
    if (r0 < r1) load_round(r0);

    for (int j = tid; j < Ng; j += BLOCK) { Es[j] = P.Ef[j]; hist[j] = 0ull; }
    if (fused) stage_total(P, S, Tt);
    if (cum_staged) {
        const float* __restrict__ g = P.cum[S];
        for (int j = tid; j < NGRID * np; j += BLOCK) Ct[j] = g[j];
    }
    if (tid == 0) {
        sh.absorbed[0] = sh.absorbed[1] = 0u; sh.removed = 0u; sh.psteps = 0u; sh.nonfinite = 0u; sh.wtries = 0u;
        sh.jsum = 0ull;
    }
    if (fused && tid < MAXPROC) sh.events[tid] = 0u;
    __syncthreads();

    unsigned psteps = 0, nabs0 = 0, nabs1 = 0, nnf = 0, wemax = 0, wtries = 0, wnumax = 0;
    long long jacc = 0;   // conduction current: sum of trunc(256 v_x^{n+1/2}) (exact)
    unsigned nrec = 0;    // warp-uniform: records of this warp so far
    unsigned qn = 0;      // warp-uniform: queued candidates

    // The first m (<= 32) queued candidates, one per lane: the candidate's
    // stream at this step (block 0) draws its next free flight (word 0) and
    // the real/null test (word 1 against the total rate at the particle's
    // energy; ions: relative to a target from the gas Maxwellian); records go
    // to the warp's list in slot order, two uint4 each: electrons {slot, id,
    // x, vx}{vy, vz, -, -}, ions {slot, id, vx, vy}{vz, w1, w2, w3} (the real
    // collisions; with the ion filter in its own kernel, every ion candidate).
    auto flush = [&](unsigned m) {
        const bool has = (unsigned)lane < m;
        const unsigned slot = has ? qs[lane] : 0u;
        const float cx = has ? qx[lane] : 0.0f, cvx = has ? qv[lane] : 0.0f;
        uint32_t id = 0u;
        float cvy = 0.0f, cvz = 0.0f;
        if (has) { id = ID[slot]; cvy = VY[slot]; cvz = VZ[slot]; }
        bool rec = false;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (has) {
            w = philox_id(pre, id);
            TC[slot] = step_lo + sub * (1u + flight_gap(w.x, inv_lnq, kcap));
            if (S == SP_E) rec = electron_is_real(P, Tt, w.y, cvx, cvy, cvz, wemax, wnumax);
            else rec = !fused || ion_is_real<S>(P, Tt, step, id, w, cvx, cvy, cvz, wtries, wemax, wnumax);
        }
        const unsigned cm = __ballot_sync(0xffffffffu, rec);
        if (rec) {
            const size_t q = r0 + nrec + __popc(cm & lt_mask);
            if (S == SP_E) {
                CAND[2 * q] = make_uint4(slot, id, __float_as_uint(cx), __float_as_uint(cvx));
                CAND[2 * q + 1] = make_uint4(__float_as_uint(cvy), __float_as_uint(cvz), 0u, 0u);
            } else {
                CAND[2 * q] = make_uint4(slot, id, __float_as_uint(cvx), __float_as_uint(cvy));
                CAND[2 * q + 1] = make_uint4(__float_as_uint(cvz), w.y, w.z, w.w);
            }
        }
        nrec += __popc(cm);
    };

    for (unsigned g0 = r0; g0 < r1; g0 += ROUND) {
        if (g0 != r0) load_round(g0);
#pragma unroll PUSH_UNROLL
        for (int k = 0; k < 4; ++k) {
            const unsigned i = g0 + 32u * k + lane;
            float x = xs[k], vx = vxs[k];
            bool cand = false;
            int dcell = -1;                  // cell deposited into (-1: none)
            unsigned long long dval = 0ull;
            if (!is_dead(x)) {
                int j; float frac;
                cell_of(x, inv_dx, Nc, j, frac);
                const float Ep = fmaf(frac, Es[j + 1] - Es[j], Es[j]);
                vx = fmaf(qmdt, Ep, vx);
                x = fmaf(vx, dts, x);
                ++psteps;
                jacc += (long long)(vx * 256.0f);   // exact scaling by 2^8, then truncation
                if (x < 0.0f) { ++nabs0; x = dead_marker(); }
                else if (x >= Lf) { ++nabs1; x = dead_marker(); }
                else if (!(x >= 0.0f) || !isfinite(vx)) { ++nnf; x = dead_marker(); }
                else {
                    // CIC deposit as (count, sum of r) per cell: node c gets
                    // 2^16 count_c - rsum_c, node c+1 gets rsum_c
                    int j2; float f2;
                    cell_of(x, inv_dx, Nc, j2, f2);
                    dcell = j2;
                    dval = (1ull << 40) + (unsigned long long)cic_r(f2);
                    if (!O2PIC_DEPOSIT_AGG) atomicAdd(&hist[j2], dval);
                    // its free flight ends at this step: a collision candidate
                    cand = (np > 0) && (tcs[k] == step_lo);
                }
                X[i] = x;
                VX[i] = vx;
            }
            if (O2PIC_DEPOSIT_AGG) {
                // the lanes of one cell add their values (peer by peer, in
                // lane order) and the lowest of them adds the sum
                const unsigned peers = __match_any_sync(0xffffffffu, dcell);
                unsigned long long sum = 0ull;
                for (unsigned m = peers; m; m &= m - 1u) sum += __shfl_sync(peers, dval, __ffs(m) - 1);
                if (dcell >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[dcell], sum);
            }
            const unsigned cm = __ballot_sync(0xffffffffu, cand);
            if (cand) {
                const unsigned q = qn + __popc(cm & lt_mask);
                qs[q] = i; qx[q] = x; qv[q] = vx;
            }
            qn += __popc(cm);
            if (qn >= 32u) {
                __syncwarp();
                flush(32u);
                const unsigned rest = qn - 32u;    // < 32: lane q moves entry 32 + q
                unsigned s0 = 0u;
                float x0 = 0.0f, v0 = 0.0f;
                if ((unsigned)lane < rest) { s0 = qs[32 + lane]; x0 = qx[32 + lane]; v0 = qv[32 + lane]; }
                __syncwarp();
                if ((unsigned)lane < rest) { qs[lane] = s0; qx[lane] = x0; qv[lane] = v0; }
                qn = rest;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (qn > 0u) flush(qn);
    unsigned nrm = 0;
    if (fused) {
        // the real collisions, by the warp that recorded them (its lanes'
        // records are visible to the whole warp after the barrier): the
        // kinematics run while other warps still push, and a removed
        // particle's charge comes off this block's histogram.  The filter
        // counted the warnings of the part it shares with the kinematics.
        __syncwarp();
        unsigned nb1 = 0, nb2 = 0, wt2 = 0, we2 = 0;
        collide_list<S, 32>(P, cum, pre, step, r0, nrec, nrec, (unsigned)lane, 0xffffffffu, lt_mask, sh.events, hist,
                            nb1, nb2, nrm, wt2, we2);
        wtries += wt2;
        if (P.births_possible[S] && lane == 0) {
            if (S == SP_E) {
                P.wcount[B_E_FROM_E][gw] = nb1;
                P.wcount[B_OM_FROM_E][gw] = nb2;
            } else if (S == SP_OM) {
                P.wcount[B_E_FROM_OM][gw] = nb2;
            }
        }
    } else if (lane == 0) {
        P.ccount[S][gw] = nrec;
    }
    pdl_trigger();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jacc += __shfl_down_sync(0xffffffffu, jacc, o);
    if (lane == 0 && jacc) atomicAdd(&sh.jsum, (unsigned long long)jacc);
    if (psteps) atomicAdd(&sh.psteps, psteps);
    if (nabs0) atomicAdd(&sh.absorbed[0], nabs0);
    if (nabs1) atomicAdd(&sh.absorbed[1], nabs1);
    if (nabs0 + nabs1 + nnf + nrm) atomicAdd(&sh.removed, nabs0 + nabs1 + nnf + nrm);
    if (nnf) atomicAdd(&sh.nonfinite, nnf);
    if (wtries) atomicAdd(&sh.wtries, wtries);
    if (wemax) atomicAdd(&C->cnt.warn_emax, (unsigned long long)wemax);
    if (wnumax) atomicAdd(&C->cnt.warn_numax, (unsigned long long)wnumax);
    __syncthreads();
    if (fused && tid < np && sh.events[tid]) atomicAdd(&C->cnt.events[S][tid], (unsigned long long)sh.events[tid]);
    unsigned long long* __restrict__ Qcopy = P.Qf[S] + (size_t)(blk & (QCOPIES - 1)) * Ng;
    for (int c = tid; c < Nc; c += BLOCK) {
        const unsigned long long v = hist[c];
        if (v) {
            const unsigned long long count = v >> 40, rsum = v & ((1ull << 40) - 1);
            atomicAdd(&Qcopy[c], (count << 16) - rsum);
            if (rsum) atomicAdd(&Qcopy[c + 1], rsum);
        }
    }
    if (tid == 0) {
        if (sh.absorbed[0]) atomicAdd(&C->cnt.absorbed[S][0], (unsigned long long)sh.absorbed[0]);
        if (sh.absorbed[1]) atomicAdd(&C->cnt.absorbed[S][1], (unsigned long long)sh.absorbed[1]);
        if (sh.removed) atomicAdd(&C->removed[S], (unsigned long long)sh.removed);
        if (sh.psteps) {
            atomicAdd(&C->cnt.particle_steps, (unsigned long long)sh.psteps);
            atomicAdd(&C->cnt.psteps[S], (unsigned long long)sh.psteps);
        }
        if (sh.nonfinite) atomicOr(&C->error_flags, ERR_NONFINITE);
        if (sh.wtries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh.wtries);
        if (sh.jsum) atomicAdd(&P.jring[(step & (JRING - 1)) * NSP + S], sh.jsum);
    }
}

// Free flights of the particles of species S drawn afresh at the current step
// n (after a load, or when new tables change nu_max): the first push at or
// after n plus sub K, K from word 0 of the particle's stream with tag
// TAG_FLIGHT + S at step n.
template <int S>
__global__ void k_flight_init(Params P) {
    DevCtrl* C = P.ctrl;
    const unsigned long long n = C->step;
    const unsigned cb = C->cur[S];
    const unsigned long long ns = (C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap;
    const float* __restrict__ X = P.sp[S].x[cb];
    const uint32_t* __restrict__ ID = P.sp[S].id[cb];
    uint32_t* __restrict__ TC = P.sp[S].tc[cb];
    const unsigned sub = P.sub[S];
    const uint32_t nf = (uint32_t)((n + sub - 1) / sub * sub);
    const PhiloxPre pre = philox_pre((uint32_t)n, TAG_FLIGHT + (uint32_t)S, (uint32_t)(n >> 32), P.seed);
    const float inv_lnq = P.inv_lnq[S], kcap = P.kcap[S];
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < ns;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (is_dead(X[i])) continue;
        TC[i] = nf + sub * flight_gap(philox_id(pre, ID[i]).x, inv_lnq, kcap);
    }
}

// Filter of the ion candidates of one species (one warp per warp of the
// particle kernel, walking its candidate list in slot order): the target
// sampled from the gas Maxwellian, the relative energy and the total rate
// against u1 nu_max, the same arithmetic as the start of collide().  It reads
// the records only (they carry the velocities and the Philox words).  The
// real collisions keep their records, compacted in place at the start of the
// list (a record is written only over one already read), and the list length
// becomes their number.  This kernel carries no kinematics, so it runs at a
// far higher occupancy than the kinematics kernel, which then sees only the
// real collisions.
template <int S>
__device__ __forceinline__ void filter_body(const Params& P, unsigned blk, unsigned nblk) {
    __shared__ float tot[NGRID];
    __shared__ unsigned sh_wtries, sh_wemax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (tid == 0) { sh_wtries = 0u; sh_wemax = 0u; }
    stage_total(P, S, tot);
    __syncthreads();
    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const unsigned nslots = (unsigned)((C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap);
    uint4* CAND = P.cand[S];
    const unsigned W = P.push_warps[S];
    const unsigned R = warp_range_len(nslots, W);
    const float numax = P.numax[S], kap = P.kappa[S], sig = P.sig_gas;
    unsigned wtries = 0, wemax = 0, wnumax = 0;
    for (unsigned gw = blk * WARPS + warp; gw < W; gw += nblk * WARPS) {
        const unsigned r0 = (gw * (unsigned long long)R < nslots) ? gw * R : nslots;
        const unsigned n = P.ccount[S][gw];
        unsigned nreal = 0;   // warp-uniform
        for (unsigned c0 = 0; c0 < n; c0 += 64) {
            uint4 a[2], b[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const unsigned ci = c0 + 32u * k + lane;
                const bool in = ci < n;
                a[k] = in ? CAND[2 * (size_t)(r0 + ci)] : make_uint4(0u, 0u, 0u, 0u);
                b[k] = in ? CAND[2 * (size_t)(r0 + ci) + 1] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (c0 + 32u * k >= n) break;   // warp-uniform
                const bool in = c0 + 32u * k + lane < n;
                bool real = false;
                if (in) {
                    Stream st;
                    st.resume(a[k].y, P.seed, step, SpeciesTraits<S>::tag, make_uint4(a[k].y, b[k].y, b[k].z, b[k].w), 1);
                    const float u1 = uniform(st.next());
                    float vtx, vty, vtz;
                    maxwellian(st, sig, vtx, vty, vtz, wtries);
                    const float gx = __uint_as_float(a[k].z) - vtx, gy = __uint_as_float(a[k].w) - vty,
                                gz = __uint_as_float(b[k].x) - vtz;
                    const float E = kap * dot3(gx, gy, gz, gx, gy, gz);
                    int i; float w; bool above;
                    grid_locate(E, i, w, above);
                    if (above) ++wemax;
                    const float total = grid_interp(tot, 1, 0, i, w);
                    if (total > numax) ++wnumax;   // above a capped majorant
                    real = (u1 * numax) < total;
                }
                const unsigned m = __ballot_sync(0xffffffffu, real);
                if (real) {
                    const size_t q = r0 + nreal + __popc(m & lt_mask);
                    CAND[2 * q] = a[k];
                    CAND[2 * q + 1] = b[k];
                }
                nreal += __popc(m);
            }
        }
        if (lane == 0) P.ccount[S][gw] = nreal;
    }
    pdl_trigger();
    if (wtries) atomicAdd(&sh_wtries, wtries);
    if (wemax) atomicAdd(&sh_wemax, wemax);
    if (wnumax) atomicAdd(&C->cnt.warn_numax, (unsigned long long)wnumax);
    __syncthreads();
    if (tid == 0) {
        if (sh_wtries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh_wtries);
        if (sh_wemax) atomicAdd(&C->cnt.warn_emax, (unsigned long long)sh_wemax);
    }
}

// Real collisions of one ion species for this step (the electrons' run at
// the end of their particle kernel).  Each warp takes two lists of the
// particle kernel's warps at once, one per half-warp (16 lanes; a list holds
// a few records at the method's rates), and walks them in slot order, 16
// records per pass through the kinematics, so the lists of a step run in one
// wave of resident warps.  Births are ranked with ballots within the
// half-warp and staged at the particle warp's slot range with their count.
constexpr int SEG = 16;
constexpr int SEGS = 32 / SEG;

template <int S>
__device__ __forceinline__ void cand_body(const Params& P, unsigned blk, unsigned nblk) {
    __shared__ unsigned events[MAXPROC];
    __shared__ unsigned sh_removed, sh_wtries, sh_wemax;
    const int np = P.nproc[S];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned seg = (unsigned)lane / SEG, sl = (unsigned)lane % SEG;
    const unsigned seg_mask = ((1u << SEG) - 1u) << (seg * SEG);
    const unsigned lt_mask = ((1u << lane) - 1u) & seg_mask;   // lanes below, same half-warp
    if (tid < MAXPROC) events[tid] = 0u;
    if (tid == 0) { sh_removed = 0u; sh_wtries = 0u; sh_wemax = 0u; }
    __syncthreads();

    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const unsigned nslots = (unsigned)((C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap);
    const bool births = P.births_possible[S] != 0;
    unsigned* cnt1 = (S == SP_E) ? P.wcount[B_E_FROM_E] : nullptr;
    unsigned* cnt2 = (S == SP_E) ? P.wcount[B_OM_FROM_E] : (S == SP_OM ? P.wcount[B_E_FROM_OM] : nullptr);
    const unsigned W = P.push_warps[S];
    const unsigned R = warp_range_len(nslots, W);
    const PhiloxPre pre = philox_pre((uint32_t)step, SpeciesTraits<S>::tag, (uint32_t)(step >> 32), P.seed);
    unsigned wtries = 0, wemax = 0, nremoved = 0;

    for (unsigned gb = (blk * WARPS + warp) * SEGS; gb < W; gb += nblk * WARPS * SEGS) {
        const unsigned gw = gb + seg;                  // this half-warp's list
        const bool valid = gw < W;
        const unsigned r0 = !valid ? 0u : ((gw * (unsigned long long)R < nslots) ? gw * R : nslots);
        const unsigned n = valid ? P.ccount[S][gw] : 0u;
        const unsigned nmax = max(n, __shfl_xor_sync(0xffffffffu, n, SEG));
        unsigned nb1 = 0, nb2 = 0;   // half-warp-uniform
        collide_list<S, SEG>(P, P.cum[S], pre, step, r0, n, nmax, sl, seg_mask, lt_mask, events, nullptr, nb1, nb2,
                             nremoved, wtries, wemax);
        if (births && valid && sl == 0) {
            if (cnt1) cnt1[gw] = nb1;
            if (cnt2) cnt2[gw] = nb2;
        }
    }
    pdl_trigger();
    if (nremoved) atomicAdd(&sh_removed, nremoved);
    if (wtries) atomicAdd(&sh_wtries, wtries);
    if (wemax) atomicAdd(&sh_wemax, wemax);
    __syncthreads();
    if (tid < np && events[tid]) atomicAdd(&C->cnt.events[S][tid], (unsigned long long)events[tid]);
    if (tid == 0) {
        if (sh_removed) atomicAdd(&C->removed[S], (unsigned long long)sh_removed);
        if (sh_wtries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh_wtries);
        if (sh_wemax) atomicAdd(&C->cnt.warn_emax, (unsigned long long)sh_wemax);
    }
}

template <int S>
constexpr int push_min_blocks() { return S == SP_E ? O2PIC_PUSH_E_MIN_BLOCKS : O2PIC_PUSH_MIN_BLOCKS; }

template <int S>
__global__ void __launch_bounds__(BLOCK, push_min_blocks<S>()) k_push(Params P) {
    pdl_wait();
    push_body<S>(P, blockIdx.x, gridDim.x);
}

template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_CAND_MIN_BLOCKS) k_cand(Params P) {
    pdl_wait();
    cand_body<S>(P, blockIdx.x, gridDim.x);
}

// The ion filter is light (no kinematics): more resident blocks per SM.
#ifndef O2PIC_FILTER_MIN_BLOCKS
#define O2PIC_FILTER_MIN_BLOCKS 3
#endif
template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_FILTER_MIN_BLOCKS) k_filter(Params P) {
    pdl_wait();
    filter_body<S>(P, blockIdx.x, gridDim.x);
}

// Batched launches: block b works for discharge map[b].x as its block
// map[b].y of map[b].z, with that discharge's parameters copied to shared
// memory (load_params).
template <int S>
__global__ void __launch_bounds__(BLOCK, push_min_blocks<S>()) k_push_b(const Params* __restrict__ all,
                                                                        const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    const uint4 m = map[blockIdx.x];
    load_params(sP, all + m.x);
    push_body<S>(sP, m.y, m.z);
}

template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_CAND_MIN_BLOCKS) k_cand_b(const Params* __restrict__ all,
                                                                        const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    const uint4 m = map[blockIdx.x];
    load_params(sP, all + m.x);
    if (sP.nproc[S] == 0) return;   // block-uniform
    cand_body<S>(sP, m.y, m.z);
}

template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_FILTER_MIN_BLOCKS) k_filter_b(const Params* __restrict__ all,
                                                                            const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    const uint4 m = map[blockIdx.x];
    load_params(sP, all + m.x);
    if (sP.nproc[S] == 0) return;   // block-uniform
    filter_body<S>(sP, m.y, m.z);
}

// Deposit of all live particles of one species into Qf (used after a load).
template <int S>
__global__ void __launch_bounds__(BLOCK) k_deposit(Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned* hist = reinterpret_cast<unsigned*>(smem);
    const int Ng = P.Ng, Nc = P.Nc;
    DevCtrl* C = P.ctrl;
    const unsigned cb = C->cur[S];
    const unsigned long long n = C->slots[S];
    const float* X = P.sp[S].x[cb];
    for (int j = threadIdx.x; j < Ng; j += BLOCK) hist[j] = 0u;
    __syncthreads();
    // each block deposits at most 2^16 - 1 particles between flushes
    const unsigned long long per = (unsigned long long)gridDim.x * BLOCK;
    unsigned long long count = 0;
    for (unsigned long long b = (unsigned long long)blockIdx.x * BLOCK; b < n; b += per) {
        const unsigned long long i = b + threadIdx.x;
        if (i < n) {
            const float x = X[i];
            if (!is_dead(x)) deposit_add(hist, x, P.inv_dx, Nc);
        }
        count += BLOCK;
        if (count >= 65536ull - BLOCK) {
            __syncthreads();
            flush_hist(hist, P.Qf[S], Ng);
            __syncthreads();
            count = 0;
        }
    }
    __syncthreads();
    flush_hist(hist, P.Qf[S], Ng);
}

}  // namespace

size_t push_smem_bytes(int species, const Params& P) {
    const size_t base = align16(align16(sizeof(PushShared)) + sizeof(float) * P.Ng) +
                        sizeof(unsigned long long) * P.Ng + sizeof(PushQueue);
    if (!(species == SP_E || O2PIC_FUSE_IONS)) return base;
    const size_t table = P.cum_smem[species] ? sizeof(float) * NGRID * (size_t)P.nproc[species] : 0;
    return base + sizeof(float) * NGRID + table;
}

bool ions_fused() { return O2PIC_FUSE_IONS != 0; }

bool cum_smem_allowed() { return O2PIC_CUM_SMEM != 0; }

void launch_flight_init(int species, const Params& P, cudaStream_t s) {
    const unsigned long long cap = P.sp[species].cap;
    const int grid = (int)(cap / 256 + 1 < 4096 ? cap / 256 + 1 : 4096);
    if (species == SP_E) k_flight_init<SP_E><<<grid, 256, 0, s>>>(P);
    else if (species == SP_OM) k_flight_init<SP_OM><<<grid, 256, 0, s>>>(P);
    else k_flight_init<SP_OP><<<grid, 256, 0, s>>>(P);
}

void launch_push(int species, const Params& P, int grid, cudaStream_t s) {
    const size_t sm = push_smem_bytes(species, P);
    if (species == SP_E) launch_pdl(k_push<SP_E>, grid, BLOCK, sm, s, P);
    else if (species == SP_OM) launch_pdl(k_push<SP_OM>, grid, BLOCK, sm, s, P);
    else launch_pdl(k_push<SP_OP>, grid, BLOCK, sm, s, P);
}

void launch_push_batched(int species, const Params* all, const uint4* map, int nblocks, size_t smem, cudaStream_t s) {
    if (species == SP_E) launch_pdl(k_push_b<SP_E>, nblocks, BLOCK, smem, s, all, map);
    else if (species == SP_OM) launch_pdl(k_push_b<SP_OM>, nblocks, BLOCK, smem, s, all, map);
    else launch_pdl(k_push_b<SP_OP>, nblocks, BLOCK, smem, s, all, map);
}

void launch_cand_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s) {
    if (species == SP_OM) launch_pdl(k_cand_b<SP_OM>, nblocks, BLOCK, 0, s, all, map);
    else if (species == SP_OP) launch_pdl(k_cand_b<SP_OP>, nblocks, BLOCK, 0, s, all, map);
}

void launch_filter(int species, const Params& P, int grid, cudaStream_t s) {
    if (species == SP_OM) launch_pdl(k_filter<SP_OM>, grid, BLOCK, 0, s, P);
    else if (species == SP_OP) launch_pdl(k_filter<SP_OP>, grid, BLOCK, 0, s, P);
}

void launch_filter_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s) {
    if (species == SP_OM) launch_pdl(k_filter_b<SP_OM>, nblocks, BLOCK, 0, s, all, map);
    else if (species == SP_OP) launch_pdl(k_filter_b<SP_OP>, nblocks, BLOCK, 0, s, all, map);
}

void launch_cand(int species, const Params& P, int grid, cudaStream_t s) {
    if (species == SP_OM) launch_pdl(k_cand<SP_OM>, grid, BLOCK, 0, s, P);
    else if (species == SP_OP) launch_pdl(k_cand<SP_OP>, grid, BLOCK, 0, s, P);
}

void launch_deposit(int species, const Params& P, int grid, cudaStream_t s) {
    const size_t sm = sizeof(unsigned) * (size_t)P.Ng;
    if (species == SP_E) k_deposit<SP_E><<<grid, BLOCK, sm, s>>>(P);
    else if (species == SP_OM) k_deposit<SP_OM><<<grid, BLOCK, sm, s>>>(P);
    else k_deposit<SP_OP><<<grid, BLOCK, sm, s>>>(P);
}

// Opt every particle kernel into the shared memory it needs (once per device).
cudaError_t configure_push_smem(size_t max_bytes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_push<SP_E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_push<SP_OM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_push<SP_OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_push_b<SP_E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_push_b<SP_OM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_push_b<SP_OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_deposit<SP_E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_deposit<SP_OM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes))) return e;
    return cudaFuncSetAttribute(k_deposit<SP_OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes);
}

int push_occupancy(int species, const Params& P, int* blocks_per_sm) {
    const size_t sm = push_smem_bytes(species, P);
    cudaError_t e;
    if (species == SP_E) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<SP_E>, BLOCK, sm);
    else if (species == SP_OM) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<SP_OM>, BLOCK, sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<SP_OP>, BLOCK, sm);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace o2
