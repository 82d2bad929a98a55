// Particle kernel of one species for one time step (Sec. 2 of the paper):
// field gather, leapfrog push in x (v_x accelerated, v_y and v_z carried),
// absorbing electrodes, null-collision Monte Carlo against the O2 / O2(a)
// background, births, and the CIC charge deposit of the pushed particles.
//
// Layout and flow (GB300-first):
//   * SoA FP32 arrays x, vx, vy, vz + u32 id, updated IN PLACE: a particle
//     keeps its slot, removed particles are marked (x = NaN) and dropped by a
//     periodic stable compaction, births are appended after the last slot.
//     The common path reads x, vx, id (12 B) and writes x, vx (8 B); vy, vz
//     are read only for collision candidates.
//   * a persistent grid; each warp owns one contiguous, 128-aligned slot range
//     and walks it in rounds of 128 (lane l takes slots l, l+32, l+64, l+96:
//     every load and store is one coalesced 128-byte line per array).  No
//     block-wide barrier between the set-up and the final flush.
//   * the gather field and the deposit live in shared memory; the deposit is
//     one 64-bit atomic per particle holding (count, sum of CIC weights) per
//     cell, turned into node charges when the block flushes;
//   * one Philox block per particle per step decides "collision candidate";
//     candidates are queued per warp in slot order and filtered 32 at a time
//     (electrons: energy against the total rate); only real collisions reach
//     the out-of-line kinematics, again 32 at a time;
//   * births are ranked with warp ballots and staged at the warp's range;
//     the end-of-step kernel places them in parent order.
#include "common.cuh"

// Launch shape of the particle kernels: minimum resident blocks per SM (caps
// the registers; 4 timed fastest of 2, 3, 4 on the 512-cell, 1.6e7-particle
// workload) and unrolling of the four particles a lane handles per round.
#ifndef O2PIC_PUSH_MIN_BLOCKS
#define O2PIC_PUSH_MIN_BLOCKS 4
#endif
#ifndef O2PIC_PUSH_UNROLL
#define O2PIC_PUSH_UNROLL 4
#endif
// Minimum resident blocks per SM of the collision kernel (caps its registers;
// 2 timed fastest of 1-4 on the same workload).
#ifndef O2PIC_CAND_MIN_BLOCKS
#define O2PIC_CAND_MIN_BLOCKS 2
#endif

namespace o2 {

namespace {

template <int S> struct SpeciesTraits;
template <> struct SpeciesTraits<SP_E> { static constexpr uint32_t tag = TAG_E; };
template <> struct SpeciesTraits<SP_OM> { static constexpr uint32_t tag = TAG_OM; };
template <> struct SpeciesTraits<SP_OP> { static constexpr uint32_t tag = TAG_OP; };

constexpr int WARPS = BLOCK / 32;           // 8
constexpr int ROUND = 128;                  // slots per warp round (4 per lane)
constexpr int Q2 = 64;                      // per-warp real-collision queue (31 + 32 max)
constexpr int PUSH_UNROLL = O2PIC_PUSH_UNROLL;

struct PushShared {
    unsigned long long jsum;     // block's sum of trunc(256 v_x^{n+1/2})
    unsigned absorbed[2];
    unsigned removed;
    unsigned psteps;
    unsigned nonfinite;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// One candidate through process selection and kinematics, exactly in the
// order of the oracle.  Returns the event index (-1 = null collision).
// bkind: 0 none, 1 ionization (two births), 2 attachment / detachment (one).
template <int S>
__device__ __noinline__ int collide(const Params& P, const float* cum, int np, unsigned long long step,
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
        maxwellian(st, P.sig_gas, vtx, vty, vtz, warn_tries);
        gx = vx - vtx; gy = vy - vty; gz = vz - vtz;
    }
    const float E = P.kappa[S] * dot3(gx, gy, gz, gx, gy, gz);
    int i; float w; bool above;
    grid_locate(E, i, w, above);
    if (above) ++warn_emax;
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

// Stage-A filter of an electron candidate: is it a real collision?  The
// same arithmetic as the start of collide(): energy of the particle, the
// total rate on the table grid and the comparison with u1 nu_max.
__device__ __forceinline__ bool electron_is_real(const Params& P, const float* __restrict__ cum, int np, uint4 w0,
                                                 float vx, float vy, float vz) {
    const float u1 = uniform(w0.y);
    const float E = P.kappa[SP_E] * dot3(vx, vy, vz, vx, vy, vz);
    int i; float w; bool above;
    grid_locate(E, i, w, above);
    return (u1 * P.numax[SP_E]) < grid_interp(cum, np, np - 1, i, w);
}

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
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;

    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const unsigned cb = C->cur[S];
    const unsigned nslots = (unsigned)((C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap);
    float* __restrict__ X = P.sp[S].x[cb];
    float* __restrict__ VX = P.sp[S].vx[cb];
    const uint32_t* __restrict__ ID = P.sp[S].id[cb];
    uint4* __restrict__ CAND = P.cand[S];
    const float qmdt = P.qmdt[S], dts = P.dt_s[S], inv_dx = P.inv_dx, Lf = P.Lf, pmax = P.pmax[S];
    const int Nc = P.Nc, Ng = P.Ng;
    const uint32_t seed = P.seed, tag = SpeciesTraits<S>::tag;
    const uint32_t step_lo = (uint32_t)step, step_hi = (uint32_t)(step >> 32);

    for (int j = tid; j < Ng; j += BLOCK) { Es[j] = P.Ef[j]; hist[j] = 0ull; }
    if (tid == 0) { sh.absorbed[0] = sh.absorbed[1] = 0u; sh.removed = 0u; sh.psteps = 0u; sh.nonfinite = 0u; sh.jsum = 0ull; }
    __syncthreads();

    // this warp's contiguous slot range
    const unsigned W = nblk * WARPS;
    const unsigned gw = blk * WARPS + warp;
    const unsigned R = warp_range_len(nslots, W);
    const unsigned r0 = (gw * (unsigned long long)R < nslots) ? gw * R : nslots;
    const unsigned r1 = (r0 + R < nslots) ? r0 + R : nslots;

    unsigned psteps = 0, nabs0 = 0, nabs1 = 0, nnf = 0;
    long long jacc = 0;   // conduction current: sum of trunc(256 v_x^{n+1/2}) (exact)
    unsigned ncand = 0;   // warp-uniform: candidates of this warp so far
    for (unsigned g0 = r0; g0 < r1; g0 += ROUND) {
        const bool full = g0 + ROUND <= r1;
        float xs[4], vxs[4];
        uint32_t ids[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned i = g0 + 32u * k + lane;
            const bool inr = full || i < r1;
            xs[k] = inr ? X[i] : dead_marker();
            vxs[k] = inr ? VX[i] : 0.0f;
            ids[k] = inr ? ID[i] : 0u;
        }
#pragma unroll PUSH_UNROLL
        for (int k = 0; k < 4; ++k) {
            const unsigned i = g0 + 32u * k + lane;
            float x = xs[k];
            bool cand = false;
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (!is_dead(x)) {
                float vx = vxs[k];
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
                    atomicAdd(&hist[j2], (1ull << 40) + (unsigned long long)cic_r(f2));
                    if (np > 0) {
                        w = philox4x32_10(make_uint4(step_lo, tag, 0u, step_hi), make_uint2(ids[k], seed));
                        cand = uniform(w.x) < pmax;
                    }
                }
                X[i] = x;
                VX[i] = vx;
            }
            // candidates go to the warp's list in slot order: {slot, w1, w2, w3}
            const unsigned cm = __ballot_sync(0xffffffffu, cand);
            if (cand) CAND[r0 + ncand + __popc(cm & lt_mask)] = make_uint4(i, w.y, w.z, w.w);
            ncand += __popc(cm);
        }
    }
    pdl_trigger();
    if (lane == 0) P.ccount[S][gw] = ncand;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jacc += __shfl_down_sync(0xffffffffu, jacc, o);
    if (lane == 0 && jacc) atomicAdd(&sh.jsum, (unsigned long long)jacc);
    if (psteps) atomicAdd(&sh.psteps, psteps);
    if (nabs0) atomicAdd(&sh.absorbed[0], nabs0);
    if (nabs1) atomicAdd(&sh.absorbed[1], nabs1);
    if (nabs0 + nabs1 + nnf) atomicAdd(&sh.removed, nabs0 + nabs1 + nnf);
    if (nnf) atomicAdd(&sh.nonfinite, nnf);
    __syncthreads();
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
        if (sh.jsum) atomicAdd(&P.jring[(step & (JRING - 1)) * NSP + S], sh.jsum);
    }
}

// Collision candidates of one species for this step: one warp per warp of
// the particle kernel, walking that warp's candidate list in slot order.
// Electrons are first filtered 32 at a time (energy against the total rate);
// the real collisions, and all ion candidates, go through the out-of-line
// kinematics 32 at a time.  Births are ranked with ballots and staged at the
// particle warp's slot range with their count.
template <int S>
__device__ __forceinline__ void cand_body(const Params& P, unsigned blk, unsigned nblk) {
    __shared__ unsigned events[MAXPROC];
    __shared__ unsigned sh_removed, sh_wtries, sh_wemax;
    __shared__ uint4 q2w_all[WARPS][Q2];
    __shared__ unsigned q2s_all[WARPS][Q2];
    __shared__ float4 q2v_all[WARPS][Q2];     // x, vx, vy, vz of the queued particle
    const int np = P.nproc[S];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint4* q2w = q2w_all[warp];
    unsigned* q2s = q2s_all[warp];
    float4* q2v = q2v_all[warp];
    const float* __restrict__ cum = P.cum[S];
    if (tid < MAXPROC) events[tid] = 0u;
    if (tid == 0) { sh_removed = 0u; sh_wtries = 0u; sh_wemax = 0u; }
    __syncthreads();

    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const unsigned cb = C->cur[S];
    const unsigned nslots = (unsigned)((C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap);
    float* __restrict__ X = P.sp[S].x[cb];
    float* __restrict__ VX = P.sp[S].vx[cb];
    float* __restrict__ VY = P.sp[S].vy[cb];
    float* __restrict__ VZ = P.sp[S].vz[cb];
    const uint32_t* __restrict__ ID = P.sp[S].id[cb];
    const uint4* __restrict__ CAND = P.cand[S];
    const float inv_dx = P.inv_dx;
    const int Nc = P.Nc;
    const bool births = P.births_possible[S] != 0;
    unsigned* cnt1 = (S == SP_E) ? P.wcount[B_E_FROM_E] : nullptr;
    unsigned* cnt2 = (S == SP_E) ? P.wcount[B_OM_FROM_E] : (S == SP_OM ? P.wcount[B_E_FROM_OM] : nullptr);
    const unsigned W = P.push_warps[S];
    const unsigned R = warp_range_len(nslots, W);
    unsigned wtries = 0, wemax = 0, nremoved = 0;

    for (unsigned gw = blk * WARPS + warp; gw < W; gw += nblk * WARPS) {
        const unsigned r0 = (gw * (unsigned long long)R < nslots) ? gw * R : nslots;
        const unsigned n = P.ccount[S][gw];
        unsigned q2n = 0, nb1 = 0, nb2 = 0;   // warp-uniform

        // kinematics of lane's particle (has = lane holds one), births ranked
        auto run_real = [&](bool has, unsigned slot, uint4 w0, float x, float vx, float vy, float vz) {
            int bkind = 0;
            float4 b1 = make_float4(0.f, 0.f, 0.f, 0.f), b2 = b1;
            if (has) {
                const uint32_t id = w0.x;   // word 0 (the candidate draw) is spent: it carries the id
                bool alive;
                const int k = collide<S>(P, cum, np, step, id, w0, x, vx, vy, vz, alive, bkind, b1, b2, wtries, wemax);
                if (k >= 0) {
                    atomicAdd(&events[k], 1u);
                    if (alive) {
                        VX[slot] = vx; VY[slot] = vy; VZ[slot] = vz;
                    } else {
                        X[slot] = dead_marker();
                        deposit_sub_global(P.Qf[S], x, inv_dx, Nc);
                        ++nremoved;
                    }
                }
            }
            if (births) {
                const unsigned m1 = __ballot_sync(0xffffffffu, bkind == 1);
                const unsigned m2 = __ballot_sync(0xffffffffu, bkind == 2);
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
        };

        auto run_queue = [&](unsigned m) {
            const bool has = (unsigned)lane < m;
            const float4 v = has ? q2v[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            run_real(has, has ? q2s[lane] : 0u, has ? q2w[lane] : make_uint4(0u, 0u, 0u, 0u), v.x, v.y, v.z, v.w);
        };
        // 128 candidates per pass, four per lane, all their loads in flight together
        for (unsigned c0 = 0; c0 < n; c0 += 128) {
            unsigned slot[4];
            uint4 w0[4];
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned ci = c0 + 32u * k + lane;
                if (ci < n) {
                    const uint4 e = CAND[r0 + ci];
                    slot[k] = e.x;
                    w0[k] = make_uint4(0u, e.y, e.z, e.w);
                } else {
                    slot[k] = 0xFFFFFFFFu;
                    w0[k] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned sl = slot[k];
                const bool in = sl != 0xFFFFFFFFu;
                v[k] = in ? make_float4(X[sl], VX[sl], VY[sl], VZ[sl]) : make_float4(0.f, 0.f, 0.f, 0.f);
                w0[k].x = in ? ID[sl] : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (c0 + 32u * k >= n) break;          // warp-uniform
                const bool in = slot[k] != 0xFFFFFFFFu;
                if (S != SP_E) {
                    // ion candidates all need the target sample: straight on
                    run_real(in, in ? slot[k] : 0u, w0[k], v[k].x, v[k].y, v[k].z, v[k].w);
                    continue;
                }
                const bool real = in && electron_is_real(P, cum, np, w0[k], v[k].y, v[k].z, v[k].w);
                const unsigned m = __ballot_sync(0xffffffffu, real);
                if (real) {
                    const unsigned q = q2n + __popc(m & lt_mask);
                    q2s[q] = slot[k]; q2w[q] = w0[k]; q2v[q] = v[k];
                }
                q2n += __popc(m);
                __syncwarp();
                if (q2n >= 32u) {
                    run_queue(32u);
                    const unsigned rest = q2n - 32u;    // < 32: lane q moves entry 32 + q
                    if ((unsigned)lane < rest) {
                        const unsigned s0 = q2s[32 + lane]; const uint4 w1 = q2w[32 + lane]; const float4 v1 = q2v[32 + lane];
                        q2s[lane] = s0; q2w[lane] = w1; q2v[lane] = v1;
                    }
                    q2n = rest;
                    __syncwarp();
                }
            }
        }
        if (q2n > 0) run_queue(q2n);
        if (births && lane == 0) {
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
__global__ void __launch_bounds__(BLOCK, O2PIC_PUSH_MIN_BLOCKS) k_push(Params P) {
    pdl_wait();
    push_body<S>(P, blockIdx.x, gridDim.x);
}

template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_CAND_MIN_BLOCKS) k_cand(Params P) {
    pdl_wait();
    cand_body<S>(P, blockIdx.x, gridDim.x);
}

// Batched launches: block b works for discharge map[b].x as its block
// map[b].y of map[b].z, with that discharge's parameters copied to shared
// memory (load_params).
template <int S>
__global__ void __launch_bounds__(BLOCK, O2PIC_PUSH_MIN_BLOCKS) k_push_b(const Params* __restrict__ all,
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
    (void)species;
    return align16(align16(sizeof(PushShared)) + sizeof(float) * P.Ng) + sizeof(unsigned long long) * P.Ng;
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
    if (species == SP_E) launch_pdl(k_cand_b<SP_E>, nblocks, BLOCK, 0, s, all, map);
    else if (species == SP_OM) launch_pdl(k_cand_b<SP_OM>, nblocks, BLOCK, 0, s, all, map);
    else launch_pdl(k_cand_b<SP_OP>, nblocks, BLOCK, 0, s, all, map);
}

void launch_cand(int species, const Params& P, int grid, cudaStream_t s) {
    if (species == SP_E) launch_pdl(k_cand<SP_E>, grid, BLOCK, 0, s, P);
    else if (species == SP_OM) launch_pdl(k_cand<SP_OM>, grid, BLOCK, 0, s, P);
    else launch_pdl(k_cand<SP_OP>, grid, BLOCK, 0, s, P);
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
