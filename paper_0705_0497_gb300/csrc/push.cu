// Particle kernel of one species for one time step (Sec. 2 of the paper):
// field gather, leapfrog push in x (v_x accelerated, v_y and v_z carried),
// absorbing electrodes, null-collision Monte Carlo against the O2 / O2(a)
// background, births, and the CIC charge deposit of the pushed particles.
//
// Layout and flow (GB300-first):
//   * SoA FP32 arrays x, vx, vy, vz + u32 id, updated IN PLACE: a particle
//     keeps its slot, removed particles are marked (x = NaN) and dropped by a
//     periodic stable compaction, births are appended after the last slot.
//     The common path reads x, vx, vy, vz, id (20 B) and writes x, vx (8 B).
//   * a persistent grid; 8192-particle tiles claimed in increasing order by
//     an atomic ticket; each thread owns 4 consecutive particles per 1024-
//     particle chunk (one 16-byte vector per array);
//   * gather field, rate tables and a fixed-point deposit histogram live in
//     shared memory; the histogram is flushed with 64-bit atomics;
//   * one Philox block per particle per step decides "collision candidate";
//     candidates go to a shared-memory queue in slot order and are processed
//     256 at a time by the whole block (no warp-divergent rare branch);
//   * births are staged per tile and placed after the tile's decoupled
//     look-back (prefix of earlier tiles' births), which keeps the order the
//     method defines (parent order) without a second pass.
#include "common.cuh"

namespace o2 {

namespace {

template <int S> struct SpeciesTraits;
template <> struct SpeciesTraits<SP_E> { static constexpr uint32_t tag = TAG_E; static constexpr int kk = KK_PUSH_E; };
template <> struct SpeciesTraits<SP_OM> { static constexpr uint32_t tag = TAG_OM; static constexpr int kk = KK_PUSH_OM; };
template <> struct SpeciesTraits<SP_OP> { static constexpr uint32_t tag = TAG_OP; static constexpr int kk = KK_PUSH_OP; };

struct PushShared {
    unsigned ws[32];
    unsigned tile;
    unsigned qn;
    unsigned long long excl;
    int ok;
    unsigned events[MAXPROC];
    unsigned absorbed[2];
    unsigned removed;
    unsigned psteps;
    unsigned warn_emax, warn_tries;
    unsigned nonfinite;
};

struct SmemLayout {
    size_t ef, hist, chist, cum, qslot, qw, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(int Ng, int Nc, int nproc, bool ion) {
    SmemLayout L;
    size_t o = align16(sizeof(PushShared));
    L.ef = o; o = align16(o + sizeof(float) * Ng);
    L.hist = o; o = align16(o + sizeof(unsigned) * Ng);
    L.chist = o; o = align16(o + (ion ? sizeof(unsigned) * Nc : 0));
    L.cum = o; o = align16(o + sizeof(float) * NGRID * (nproc > 0 ? nproc : 1));
    L.qw = o; o = align16(o + sizeof(uint4) * QCAP);
    L.qslot = o; o = align16(o + sizeof(unsigned) * QCAP);
    L.total = o;
    return L;
}

// One candidate through process selection and kinematics, exactly in the
// order of the oracle.  Returns the event index (-1 = null collision).
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
        maxwellian(st, P.sig_gas, vtx, vty, vtz, warn_tries);
        gx = vx - vtx; gy = vy - vty; gz = vz - vtz;
    }
    const float E = P.kappa[S] * dot3(gx, gy, gz, gx, gy, gz);
    int i; float w; bool above;
    grid_locate(E, i, w, above);
    if (above) ++warn_emax;
    const float target = u1 * P.numax[S];
    int k = -1;
    for (int kk = 0; kk < np; ++kk) {
        if (target < grid_interp(cum, np, kk, i, w)) { k = kk; break; }
    }
    if (k < 0) return -1;
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

__device__ __forceinline__ void deposit_sub(unsigned* hist, float x, float inv_dx, int Nc) {
    int j; float frac;
    cell_of(x, inv_dx, Nc, j, frac);
    const uint32_t r = cic_r(frac);
    atomicSub(&hist[j], 65536u - r);
    atomicSub(&hist[j + 1], r);
}

// deposit of a birth straight into the global accumulator (rare)
__device__ __forceinline__ void deposit_global(unsigned long long* Q, float x, float inv_dx, int Nc) {
    int j; float frac;
    cell_of(x, inv_dx, Nc, j, frac);
    const uint32_t r = cic_r(frac);
    atomicAdd(&Q[j], (unsigned long long)(65536u - r));
    atomicAdd(&Q[j + 1], (unsigned long long)r);
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

// Write one birth into species d at slot `slot` with id `id`.
__device__ __forceinline__ void place_birth(const Params& P, int d, unsigned long long slot, unsigned long long id64,
                                            float4 b, unsigned long long* err) {
    const SpeciesBuf& B = P.sp[d];
    if (slot >= B.cap) { atomicOr(err, ERR_CAPACITY); return; }
    if (id64 > 0xFFFFFFFFull) { atomicOr(err, ERR_ID); }
    const unsigned cb = P.ctrl->cur[d];
    B.x[cb][slot] = b.x;
    B.vx[cb][slot] = b.y;
    B.vy[cb][slot] = b.z;
    B.vz[cb][slot] = b.w;
    B.id[cb][slot] = (uint32_t)id64;
    deposit_global(P.Qb[d], b.x, P.inv_dx, P.Nc);
}

template <int S>
__global__ void __launch_bounds__(BLOCK) k_push(Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool ION = (S != SP_E);
    constexpr int KKIND = SpeciesTraits<S>::kk;
    const int np = P.nproc[S];
    const SmemLayout L = smem_layout(P.Ng, P.Nc, np, ION);
    PushShared& sh = *reinterpret_cast<PushShared*>(smem);
    float* Es = reinterpret_cast<float*>(smem + L.ef);
    unsigned* hist = reinterpret_cast<unsigned*>(smem + L.hist);
    unsigned* chist = reinterpret_cast<unsigned*>(smem + L.chist);
    float* cum = reinterpret_cast<float*>(smem + L.cum);
    uint4* qw = reinterpret_cast<uint4*>(smem + L.qw);
    unsigned* qslot = reinterpret_cast<unsigned*>(smem + L.qslot);
    const int tid = threadIdx.x;

    DevCtrl* C = P.ctrl;
    const unsigned long long step = C->step;
    const unsigned long long epoch = C->epoch;
    const unsigned cb = C->cur[S];
    const unsigned long long nslots = (C->slots[S] < P.sp[S].cap) ? C->slots[S] : P.sp[S].cap;
    const unsigned ntiles = (unsigned)ceil_div(nslots, TILE);
    float* __restrict__ X = P.sp[S].x[cb];
    float* __restrict__ VX = P.sp[S].vx[cb];
    float* __restrict__ VY = P.sp[S].vy[cb];
    float* __restrict__ VZ = P.sp[S].vz[cb];
    const uint32_t* __restrict__ ID = P.sp[S].id[cb];
    const bool track_cells = ION && P.have_neutral;
    const float qmdt = P.qmdt[S], dts = P.dt_s[S], inv_dx = P.inv_dx, Lf = P.Lf, pmax = P.pmax[S];
    const int Nc = P.Nc, Ng = P.Ng;
    const uint32_t seed = P.seed, tag = SpeciesTraits<S>::tag;

    for (int j = tid; j < Ng; j += BLOCK) { Es[j] = P.Ef[j]; hist[j] = 0u; }
    for (int i = tid; i < NGRID * np; i += BLOCK) cum[i] = P.cum[S][i];
    if (tid < MAXPROC) sh.events[tid] = 0u;
    if (tid == 0) {
        sh.absorbed[0] = sh.absorbed[1] = 0u;
        sh.removed = 0u; sh.psteps = 0u; sh.warn_emax = 0u; sh.warn_tries = 0u; sh.nonfinite = 0u;
    }
    // birth destinations (slots and ids already committed before this step)
    unsigned long long dst_slot0 = 0, dst_id0 = 0, dst2_slot0 = 0, dst2_id0 = 0;
    if (S == SP_E) {
        dst_slot0 = C->slots[SP_E];             // e from ionization
        dst_id0 = C->next_id[SP_E];
        dst2_slot0 = C->slots[SP_OM];           // O- from attachment
        dst2_id0 = C->next_id[SP_OM];
    } else if (S == SP_OM) {
        const unsigned long long before = C->births[B_E_FROM_E];
        dst_slot0 = C->slots[SP_E] + before;    // e from detachment, after the e-kernel's births
        dst_id0 = (unsigned long long)C->next_id[SP_E] + before;
    }
    const unsigned long long op_slot0 = C->slots[SP_OP];
    const unsigned long long op_id0 = C->next_id[SP_OP];
    __syncthreads();

    unsigned tiles_since_flush = 0;
    for (;;) {
        if (tid == 0) sh.tile = atomicAdd(&C->ticket[KKIND], 1u);
        __syncthreads();
        const unsigned tile = sh.tile;
        __syncthreads();
        if (tile >= ntiles) break;

        const unsigned long long base = (unsigned long long)tile * TILE;
        const unsigned long long end = (base + TILE < nslots) ? base + TILE : nslots;
        if (track_cells) for (int c = tid; c < Nc; c += BLOCK) chist[c] = 0u;
        unsigned qn = 0;            // uniform across the block
        unsigned nb1 = 0, nb2 = 0;  // births staged in this tile (uniform)
        if (tid == 0) sh.qn = 0;
        __syncthreads();

        // -------- process a batch of queued candidates (entries [0, n))
        auto run_batch = [&](unsigned n) {
            bool has = (unsigned)tid < n;
            int bkind = 0;
            float4 b1 = make_float4(0, 0, 0, 0), b2 = b1;
            if (has) {
                const unsigned slot = qslot[tid];
                const uint4 w0 = qw[tid];
                const float x = X[slot];
                float vx = VX[slot], vy = VY[slot], vz = VZ[slot];
                const uint32_t id = ID[slot];
                bool alive;
                unsigned wt = 0, we = 0;
                const int k = collide<S>(P, cum, np, step, id, w0, x, vx, vy, vz, alive, bkind, b1, b2, wt, we);
                if (wt) atomicAdd(&sh.warn_tries, wt);
                if (we) atomicAdd(&sh.warn_emax, we);
                if (k >= 0) {
                    atomicAdd(&sh.events[k], 1u);
                    if (alive) {
                        VX[slot] = vx; VY[slot] = vy; VZ[slot] = vz;
                    } else {
                        X[slot] = dead_marker();
                        deposit_sub(hist, x, inv_dx, Nc);
                        if (track_cells) { int j; float fr; cell_of(x, inv_dx, Nc, j, fr); atomicSub(&chist[j], 1u); }
                        atomicAdd(&sh.removed, 1u);
                    }
                }
            }
            if (P.births_possible[S]) {
                // ranks of this batch's births (parent order), then stage them
                const unsigned f1 = (bkind == 1) ? 1u : 0u;
                const unsigned f2 = (bkind == 2) ? 1u : 0u;
                unsigned t1, t2;
                const unsigned packed = block_excl_scan<BLOCK>(f1 | (f2 << 16), sh.ws, &t1);
                t2 = t1 >> 16; t1 &= 0xFFFFu;
                const unsigned r1 = packed & 0xFFFFu, r2 = packed >> 16;
                const unsigned long long sbase = (unsigned long long)tile * TILE;
                if (S == SP_E) {
                    if (f1) {
                        P.stage[B_E_FROM_E][sbase + nb1 + r1] = b1;
                        P.stage[B_OP_FROM_E][sbase + nb1 + r1] = b2;
                    }
                    if (f2) P.stage[B_OM_FROM_E][sbase + nb2 + r2] = b1;
                } else if (S == SP_OM) {
                    if (f2) P.stage[B_E_FROM_OM][sbase + nb2 + r2] = b1;
                }
                nb1 += t1; nb2 += t2;
            }
            __syncthreads();
        };

        for (int c = 0; c < CHUNKS_PER_TILE; ++c) {
            const unsigned long long cb0 = base + (unsigned long long)c * CHUNK;
            if (cb0 >= end) break;
            const unsigned long long i0 = cb0 + 4ull * tid;
            float x[4], vx[4], vy[4], vz[4];
            uint32_t id[4];
            const bool full = (i0 + 3 < end);
            if (full) {
                const float4 a = *reinterpret_cast<const float4*>(X + i0);
                const float4 b = *reinterpret_cast<const float4*>(VX + i0);
                const float4 cc = *reinterpret_cast<const float4*>(VY + i0);
                const float4 d = *reinterpret_cast<const float4*>(VZ + i0);
                const uint4 e = *reinterpret_cast<const uint4*>(ID + i0);
                x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
                vx[0] = b.x; vx[1] = b.y; vx[2] = b.z; vx[3] = b.w;
                vy[0] = cc.x; vy[1] = cc.y; vy[2] = cc.z; vy[3] = cc.w;
                vz[0] = d.x; vz[1] = d.y; vz[2] = d.z; vz[3] = d.w;
                id[0] = e.x; id[1] = e.y; id[2] = e.z; id[3] = e.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (i0 + k < end) {
                        x[k] = X[i0 + k]; vx[k] = VX[i0 + k]; vy[k] = VY[i0 + k]; vz[k] = VZ[i0 + k]; id[k] = ID[i0 + k];
                    } else {
                        x[k] = dead_marker(); vx[k] = vy[k] = vz[k] = 0.0f; id[k] = 0u;
                    }
                }
            }
            unsigned cand = 0u;
            uint4 wv[4];
            unsigned nabs0 = 0, nabs1 = 0, nps = 0, nnf = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                wv[k] = make_uint4(0, 0, 0, 0);
                if (is_dead(x[k])) continue;
                int j; float frac;
                cell_of(x[k], inv_dx, Nc, j, frac);
                const float Ep = fmaf(frac, Es[j + 1] - Es[j], Es[j]);
                vx[k] = fmaf(qmdt, Ep, vx[k]);
                x[k] = fmaf(vx[k], dts, x[k]);
                ++nps;
                if (x[k] < 0.0f) { ++nabs0; x[k] = dead_marker(); continue; }
                if (x[k] >= Lf) { ++nabs1; x[k] = dead_marker(); continue; }
                if (!(x[k] >= 0.0f) || !isfinite(vx[k])) { ++nnf; x[k] = dead_marker(); continue; }
                int j2; float f2;
                cell_of(x[k], inv_dx, Nc, j2, f2);
                const uint32_t r = cic_r(f2);
                atomicAdd(&hist[j2], 65536u - r);
                atomicAdd(&hist[j2 + 1], r);
                if (track_cells) atomicAdd(&chist[j2], 1u);
                if (np > 0) {
                    const uint4 w = philox4x32_10(make_uint4((uint32_t)step, tag, 0u, (uint32_t)(step >> 32)),
                                                  make_uint2(id[k], seed));
                    if (uniform(w.x) < pmax) { cand |= 1u << k; wv[k] = w; }
                }
            }
            if (full) {
                *reinterpret_cast<float4*>(X + i0) = make_float4(x[0], x[1], x[2], x[3]);
                *reinterpret_cast<float4*>(VX + i0) = make_float4(vx[0], vx[1], vx[2], vx[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (i0 + k < end) { X[i0 + k] = x[k]; VX[i0 + k] = vx[k]; }
            }
            if (nabs0) atomicAdd(&sh.absorbed[0], nabs0);
            if (nabs1) atomicAdd(&sh.absorbed[1], nabs1);
            if (nabs0 + nabs1 + nnf) atomicAdd(&sh.removed, nabs0 + nabs1 + nnf);
            if (nps) atomicAdd(&sh.psteps, nps);
            if (nnf) atomicAdd(&sh.nonfinite, nnf);

            // enqueue candidates in slot order
            unsigned total;
            const unsigned off = block_excl_scan<BLOCK>(__popc(cand), sh.ws, &total);
            if (cand) {
                unsigned q = qn + off;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (cand & (1u << k)) { qslot[q] = (unsigned)(i0 + k); qw[q] = wv[k]; ++q; }
            }
            qn += total;
            __syncthreads();
            while (qn >= (unsigned)BLOCK) {
                run_batch(BLOCK);
                // move the remaining entries to the front; entry q is read
                // (from BLOCK + q) and written (to q) by the same thread, one
                // pass after it read that slot, so no cross-thread hazard
                const unsigned rest = qn - BLOCK;
                for (unsigned q = tid; q < rest; q += BLOCK) {
                    const unsigned s0 = qslot[BLOCK + q];
                    const uint4 w0 = qw[BLOCK + q];
                    qslot[q] = s0; qw[q] = w0;
                }
                qn = rest;
                __syncthreads();
            }
        }
        if (qn > 0) run_batch(qn);

        // -------- births: prefix over earlier tiles, then place them
        if (P.births_possible[S]) {
            if (tid == 0) {
                bool ok;
                sh.excl = lookback(P.lb_flag[KKIND], P.lb_val[KKIND], tile, pack2(nb1, nb2), epoch,
                                   &C->error_flags, &ok);
                sh.ok = ok ? 1 : 0;
                if (ok && tile == ntiles - 1) {
                    const unsigned long long incl = add2(sh.excl, pack2(nb1, nb2));
                    const unsigned tot1 = (unsigned)incl, tot2 = (unsigned)(incl >> 32);
                    if (S == SP_E) {
                        C->births[B_E_FROM_E] = tot1;
                        C->births[B_OP_FROM_E] = tot1;
                        C->births[B_OM_FROM_E] = tot2;
                    } else if (S == SP_OM) {
                        C->births[B_E_FROM_OM] = tot2;
                    }
                }
            }
            __syncthreads();
            if (sh.ok) {
                const unsigned e1 = (unsigned)sh.excl, e2 = (unsigned)(sh.excl >> 32);
                const unsigned long long sbase = (unsigned long long)tile * TILE;
                if (S == SP_E) {
                    for (unsigned r = tid; r < nb1; r += BLOCK) {
                        const unsigned long long k = (unsigned long long)e1 + r;
                        place_birth(P, SP_E, dst_slot0 + k, dst_id0 + k, P.stage[B_E_FROM_E][sbase + r], &C->error_flags);
                        place_birth(P, SP_OP, op_slot0 + k, op_id0 + k, P.stage[B_OP_FROM_E][sbase + r], &C->error_flags);
                    }
                    for (unsigned r = tid; r < nb2; r += BLOCK) {
                        const unsigned long long k = (unsigned long long)e2 + r;
                        place_birth(P, SP_OM, dst2_slot0 + k, dst2_id0 + k, P.stage[B_OM_FROM_E][sbase + r], &C->error_flags);
                    }
                } else if (S == SP_OM) {
                    for (unsigned r = tid; r < nb2; r += BLOCK) {
                        const unsigned long long k = (unsigned long long)e2 + r;
                        place_birth(P, SP_E, dst_slot0 + k, dst_id0 + k, P.stage[B_E_FROM_OM][sbase + r], &C->error_flags);
                    }
                }
            }
        }
        // -------- per-tile cell counts of the surviving ions, for (17)
        if (track_cells) {
            __syncthreads();
            unsigned* H = P.hist[S == SP_OM ? 0 : 1] + (size_t)tile * Nc;
            for (int c = tid; c < Nc; c += BLOCK) H[c] = chist[c];
        }
        if (++tiles_since_flush == FLUSH_TILES) {
            __syncthreads();
            flush_hist(hist, P.Qf[S], Ng);
            tiles_since_flush = 0;
        }
        __syncthreads();
    }
    __syncthreads();
    flush_hist(hist, P.Qf[S], Ng);
    if (tid < np && sh.events[tid]) atomicAdd(&C->cnt.events[S][tid], (unsigned long long)sh.events[tid]);
    if (tid == 0) {
        if (sh.absorbed[0]) atomicAdd(&C->cnt.absorbed[S][0], (unsigned long long)sh.absorbed[0]);
        if (sh.absorbed[1]) atomicAdd(&C->cnt.absorbed[S][1], (unsigned long long)sh.absorbed[1]);
        if (sh.removed) atomicAdd(&C->removed[S], (unsigned long long)sh.removed);
        if (sh.psteps) {
            atomicAdd(&C->cnt.particle_steps, (unsigned long long)sh.psteps);
            atomicAdd(&C->cnt.psteps[S], (unsigned long long)sh.psteps);
        }
        if (sh.warn_emax) atomicAdd(&C->cnt.warn_emax, (unsigned long long)sh.warn_emax);
        if (sh.warn_tries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh.warn_tries);
        if (sh.nonfinite) atomicOr(&C->error_flags, ERR_NONFINITE);
    }
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
    return smem_layout(P.Ng, P.Nc, P.nproc[species], species != SP_E).total;
}

void launch_push(int species, const Params& P, int grid, cudaStream_t s) {
    const size_t sm = push_smem_bytes(species, P);
    if (species == SP_E) k_push<SP_E><<<grid, BLOCK, sm, s>>>(P);
    else if (species == SP_OM) k_push<SP_OM><<<grid, BLOCK, sm, s>>>(P);
    else k_push<SP_OP><<<grid, BLOCK, sm, s>>>(P);
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
