// Ion-ion neutralization (17), O- + O2+ -> O + O2, on ion steps: a binary,
// cell-local (DSMC-like) process at the post-push positions.
//
// Pairing (the reading used by the oracle): in cell c take the surviving O-
// and O2+ in array order, n- and n+ of them, m = min, M = max, and a shift
// r_c drawn per cell and step; the i-th member of the shorter list (O- on a
// tie), i < m, is paired with member (i + r_c) mod M of the longer one.  A
// pair reacts with probability P = M w sigma_n(E_rel) g dt_ion / (A dx).
//
// GPU form.  The acceptance draw u of a pair needs only the O- id, and
// P <= K_max M pf (pf = w dt_ion / (A dx)), so an O- can react only if
// u < K_max M pf; at the method's weights and time steps that bound is
// ~1e-6 and only a handful of O- per step pass it.  So:
//   * k_pair_hist counts, per 8192-slot tile of each ion species, the live
//     ions per cell, and adds them into per-cell totals n-, n+;
//   * k_pair streams x and id of the O- once, draws u and flags the O- below
//     the bound (M from the totals);
//   * for a flagged O- the whole block finds its rank k in the cell list
//     (counts of the earlier tiles + same-cell slots before it in its tile),
//     the partner rank q, the O2+ tile holding rank q (block scan of that
//     cell's per-tile counts) and the partner's slot there (block scan of the
//     hits in slot order), each step with all of the block's loads in flight;
//     one thread then does the reaction test with the exact P.
// Reactions only append (O- slot, O2+ slot) to the removal list and take the
// pair out of the fresh deposit; both are order-independent, so flagged ions
// may be resolved in any order.
//
// The kernels take the two species, tables and lists as a PairSpec: the same
// code runs (22) e + O- -> O + 2e (A = O-, B = e, only A removed; its
// kinematics and births in k_edet_apply) and (16) e + O2+ -> O + O (A = e)
// before (17) (A = O-); the removals of (22) and (16) are applied before the
// next process counts its particles.
#include "common.cuh"

namespace o2 {

namespace {

constexpr int HIST_T = 512;                  // threads of k_pair_hist
constexpr int HIST_PER = TILE / HIST_T;      // 16 slots per thread
constexpr int PAIR_T = 256;                  // threads of k_pair
constexpr int PER_T = TILE / PAIR_T;         // 32 slots of a tile per thread
constexpr int LCAP = 256;                    // flagged O- listed per tile before the slow path
constexpr unsigned short CELL_DEAD = 0x7FFFu, CELL_FLAG = 0x8000u;
static_assert(PER_T == 32, "one 32-bit hit mask per thread");
static_assert(MAX_NODES - 1 < CELL_DEAD, "cell index fits 15 bits");

// Per tile of each ion species, the live ions per cell (post-push
// positions): hist[sp][tile][cell]; and the per-cell totals ptot[sp][cell]
// (zero on entry; the end-of-step kernel clears them).  Blocks take tiles of
// O- first, then of O2+, and add their totals once at the end.
__device__ __forceinline__ void pair_hist_body(const Params& P, const PairSpec& Sp, unsigned blk, unsigned nblk) {
    extern __shared__ unsigned hsm[];   // [Nc] tile counts, [2][Nc] block totals
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    unsigned* bt = hsm + Nc;
    for (int c = threadIdx.x; c < 2 * Nc; c += HIST_T) bt[c] = 0u;
    const unsigned long long nsa = C->slots[Sp.A], nsb = C->slots[Sp.B];
    const unsigned nta = (unsigned)ceil_div(nsa, TILE), ntb = (unsigned)ceil_div(nsb, TILE);
    for (unsigned g = blk; g < nta + ntb; g += nblk) {
        const int sp = (g < nta) ? 0 : 1;
        const unsigned tile = (g < nta) ? g : g - nta;
        const int S = sp == 0 ? Sp.A : Sp.B;
        const unsigned long long n = sp == 0 ? nsa : nsb;
        const float* __restrict__ X = P.sp[S].x[C->cur[S]];
        for (int c = threadIdx.x; c < Nc; c += HIST_T) hsm[c] = 0u;
        const unsigned long long base = (unsigned long long)tile * TILE;
        float xs[HIST_PER];
#pragma unroll
        for (int i = 0; i < HIST_PER; ++i) {
            const unsigned long long p = base + (unsigned long long)i * HIST_T + threadIdx.x;
            xs[i] = (p < n) ? X[p] : dead_marker();
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < HIST_PER; ++i) {
            if (!is_dead(xs[i])) {
                int c; float fr;
                cell_of(xs[i], P.inv_dx, Nc, c, fr);
                atomicAdd(&hsm[c], 1u);
            }
        }
        __syncthreads();
        unsigned* H = (sp == 0 ? Sp.histA : Sp.histB) + (size_t)tile * Nc;
        for (int c = threadIdx.x; c < Nc; c += HIST_T) {
            const unsigned v = hsm[c];
            H[c] = v;
            bt[sp * Nc + c] += v;
        }
        __syncthreads();
    }
    pdl_trigger();
    for (int c = threadIdx.x; c < 2 * Nc; c += HIST_T)
        if (bt[c]) atomicAdd(&Sp.tot[c], bt[c]);
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned* ws) {
    unsigned total;
    (void)block_excl_scan<PAIR_T>(v, ws, &total);
    return total;
}

// Resolve one flagged O- (tile position pos, cell in cell16[pos]).  Every
// thread of the block calls it; all return at the same point except at the
// very end.  sh = 2 words of shared memory for the partner tile search.
__device__ void resolve_one(const Params& P, const PairSpec& Sp, unsigned pos, unsigned tile, unsigned long long base,
                            const unsigned short* cell16, unsigned* ws, unsigned* sh, unsigned long long step,
                            unsigned long long nsp, unsigned ntp, unsigned cm, unsigned cp, unsigned& gt1) {
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const int tid = threadIdx.x;
    const unsigned c = cell16[pos] & CELL_DEAD;
    // rank k of the O- in its cell list
    unsigned cnt = 0;
    const unsigned* H0 = Sp.histA;
    for (unsigned t = tid; t < tile; t += PAIR_T) cnt += H0[(size_t)t * Nc + c];
#pragma unroll 8
    for (int i = 0; i < PER_T; ++i) {
        const unsigned q = (unsigned)i * PAIR_T + tid;
        if (q < pos && (cell16[q] & CELL_DEAD) == c) ++cnt;
    }
    const unsigned k = block_sum(cnt, ws);
    const unsigned nm = Sp.tot[c], npl = Sp.tot[Nc + c];
    const unsigned m = nm < npl ? nm : npl, M = nm < npl ? npl : nm;
    if (m == 0 || k >= nm) return;   // block-uniform
    const uint4 wr = philox4x32_10(make_uint4((uint32_t)step, Sp.tag_shift, 0u, (uint32_t)(step >> 32)),
                                   make_uint2(c, P.seed));
    const unsigned r = wr.x % M;
    unsigned q;
    if (nm <= npl) {
        q = k + r; if (q >= M) q -= M;
    } else {
        unsigned i = k + (M - r); if (i >= M) i -= M;   // the O2+ of rank i has this O- as partner
        if (i >= m) return;                              // block-uniform
        q = i;
    }
    // O2+ tile holding rank q: thread t sums a contiguous group of tiles
    const unsigned* H1 = Sp.histB;
    const unsigned per = (ntp + PAIR_T - 1) / PAIR_T;
    const unsigned t0 = (unsigned)tid * per, t1 = (t0 + per < ntp) ? t0 + per : ntp;
    unsigned gs = 0;
    for (unsigned t = t0; t < t1; ++t) gs += H1[(size_t)t * Nc + c];
    unsigned gtot;
    const unsigned gex = block_excl_scan<PAIR_T>(gs, ws, &gtot);
    if (q >= gtot) return;   // block-uniform (inconsistent counts; never expected)
    if (gex <= q && q < gex + gs) {
        unsigned run = gex, t = t0;
        for (; t < t1; ++t) {
            const unsigned v = H1[(size_t)t * Nc + c];
            if (q < run + v) break;
            run += v;
        }
        sh[0] = t;
        sh[1] = q - run;
    }
    __syncthreads();
    const unsigned lo = sh[0], want = sh[1];
    __syncthreads();
    // the partner's slot: rank `want` among the tile's live O2+ of cell c
    const float* XP = P.sp[Sp.B].x[cp];
    const unsigned long long bb = (unsigned long long)lo * TILE + (unsigned long long)tid * PER_T;
    float xs[PER_T];
#pragma unroll
    for (int i = 0; i < PER_T; ++i) xs[i] = (bb + i < nsp) ? XP[bb + i] : dead_marker();
    unsigned mask = 0;
#pragma unroll
    for (int i = 0; i < PER_T; ++i) {
        if (!is_dead(xs[i])) {
            int j; float fr;
            cell_of(xs[i], P.inv_dx, Nc, j, fr);
            if ((unsigned)j == c) mask |= 1u << i;
        }
    }
    const unsigned h = __popc(mask);
    unsigned htot;
    const unsigned excl = block_excl_scan<PAIR_T>(h, ws, &htot);
    if (want < excl || want >= excl + h) return;
    unsigned bits = mask;
    for (unsigned t = 0; t < want - excl; ++t) bits &= bits - 1u;
    const unsigned b_slot = (unsigned)(bb + (unsigned)(__ffs(bits) - 1));
    // reaction test with the exact probability
    const unsigned long long p = base + pos;
    const SpeciesBuf& SM = P.sp[Sp.A];
    const SpeciesBuf& SPp = P.sp[Sp.B];
    const uint4 w = philox4x32_10(make_uint4((uint32_t)step, Sp.tag_pair, 0u, (uint32_t)(step >> 32)),
                                  make_uint2(SM.id[cm][p], P.seed));
    const float u = uniform(w.x);
    const float gx = SM.vx[cm][p] - SPp.vx[cp][b_slot];
    const float gy = SM.vy[cm][p] - SPp.vy[cp][b_slot];
    const float gz = SM.vz[cm][p] - SPp.vz[cp][b_slot];
    const float E = Sp.kappa * dot3(gx, gy, gz, gx, gy, gz);
    int gi; float gw; bool above;
    grid_locate(E, gi, gw, above);
    if (above) atomicAdd(&C->cnt.warn_emax, 1ull);
    const float K = grid_interp(Sp.K, 1, 0, gi, gw);
    const float Pp = K * (P.pair_factor * (float)M);
    if (Pp > 1.0f) ++gt1;
    if (u < Pp && E >= Sp.thr) {
        const unsigned idx = atomicAdd(Sp.nremovals, 1u);
        if (idx < Sp.max_removals) {
            Sp.removal[2 * idx] = (unsigned)p;
            Sp.removal[2 * idx + 1] = b_slot;
        }
        // take both out of the fresh deposit
        int j; float f;
        cell_of(SM.x[cm][p], P.inv_dx, Nc, j, f);
        uint32_t rr = cic_r(f);
        atomicAdd(&P.Qf[Sp.A][j], 0ull - (unsigned long long)(65536u - rr));
        atomicAdd(&P.Qf[Sp.A][j + 1], 0ull - (unsigned long long)rr);
        if (!Sp.b_survives) {
            cell_of(XP[b_slot], P.inv_dx, Nc, j, f);
            rr = cic_r(f);
            atomicAdd(&P.Qf[Sp.B][j], 0ull - (unsigned long long)(65536u - rr));
            atomicAdd(&P.Qf[Sp.B][j + 1], 0ull - (unsigned long long)rr);
        }
    }
}

// One block per O- tile (grid-stride): the streaming pass, then the flagged
// O- of the tile.  Block 0 also adds sum_c min(n-, n+) to the pair counter.
__device__ __forceinline__ void pair_body(const Params& P, const PairSpec& Sp, unsigned blk, unsigned nblk) {
    __shared__ unsigned short cell16[TILE];
    __shared__ unsigned short list[LCAP];
    __shared__ unsigned ws[32];
    __shared__ unsigned sh[2];
    __shared__ unsigned nflag;
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const int tid = threadIdx.x;
    const unsigned long long step = C->step;
    const unsigned long long nsm = C->slots[Sp.A], nsp = C->slots[Sp.B];
    const unsigned ntm = (unsigned)ceil_div(nsm, TILE), ntp = (unsigned)ceil_div(nsp, TILE);
    const unsigned cm = C->cur[Sp.A], cp = C->cur[Sp.B];
    const float* __restrict__ XM = P.sp[Sp.A].x[cm];
    const uint32_t* __restrict__ IDM = P.sp[Sp.A].id[cm];
    const unsigned* __restrict__ tot = Sp.tot;
    // the acceptance draw's Philox block (counter (step, tag, 0), key (id,
    // seed)) with its id-free first-round products computed once
    const PhiloxPre pre = philox_pre((uint32_t)step, Sp.tag_pair, (uint32_t)(step >> 32), P.seed);
    unsigned gt1 = 0;

    if (blk == 0) {
        unsigned pairs = 0;   // at most 2^32 ions in all
        for (int c = tid; c < Nc; c += PAIR_T) {
            const unsigned a = tot[c], b = tot[Nc + c];
            pairs += a < b ? a : b;
        }
        const unsigned s = block_sum(pairs, ws);
        if (tid == 0 && s) atomicAdd(Sp.tested, (unsigned long long)s);
    }

    for (unsigned tile = blk; tile < ntm; tile += nblk) {
        const unsigned long long base = (unsigned long long)tile * TILE;
        if (tid == 0) nflag = 0u;
        __syncthreads();
#pragma unroll
        for (int h = 0; h < PER_T; h += 16) {
            float xs[16];
            uint32_t ids[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const unsigned long long p = base + (unsigned long long)(h + i) * PAIR_T + tid;
                const bool in = p < nsm;
                xs[i] = in ? XM[p] : dead_marker();
                ids[i] = in ? IDM[p] : 0u;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const unsigned pos = (unsigned)(h + i) * PAIR_T + tid;
                unsigned short cc = CELL_DEAD;
                if (!is_dead(xs[i])) {
                    int c; float fr;
                    cell_of(xs[i], P.inv_dx, Nc, c, fr);
                    const unsigned a = __ldg(&tot[c]), b = __ldg(&tot[Nc + c]);
                    const unsigned M = a < b ? b : a;
                    const float u = uniform(philox_id(pre, ids[i]).x);
                    cc = (unsigned short)c;
                    if (u < Sp.Kmax_hi * (P.pair_factor * (float)M)) {
                        cc |= CELL_FLAG;
                        const unsigned idx = atomicAdd(&nflag, 1u);
                        if (idx < LCAP) list[idx] = (unsigned short)pos;
                    }
                }
                cell16[pos] = cc;
            }
        }
        __syncthreads();
        const unsigned nf = nflag;
        if (nf > 0 && nf <= LCAP) {
            for (unsigned j = 0; j < nf; ++j)
                resolve_one(P, Sp, list[j], tile, base, cell16, ws, sh, step, nsp, ntp, cm, cp, gt1);
        } else if (nf > LCAP) {
            // many flagged ions: list them segment by segment from the flags
            for (int seg = 0; seg < PER_T; ++seg) {
                const unsigned pos = (unsigned)seg * PAIR_T + tid;
                const bool f = (cell16[pos] & CELL_FLAG) != 0;
                unsigned ns;
                const unsigned idx = block_excl_scan<PAIR_T>(f ? 1u : 0u, ws, &ns);
                if (f) list[idx] = (unsigned short)pos;
                __syncthreads();
                for (unsigned j = 0; j < ns; ++j)
                    resolve_one(P, Sp, list[j], tile, base, cell16, ws, sh, step, nsp, ntp, cm, cp, gt1);
                __syncthreads();
            }
        }
        __syncthreads();
    }
    pdl_trigger();
    if (gt1) atomicAdd(&C->cnt.warn_pair_gt1, (unsigned long long)gt1);
}

// The removals of a pair process that runs before another (16 before 17):
// mark both particles of every listed pair dead, count them, clear the list.
__device__ __forceinline__ void pair_apply_body(const Params& P, const PairSpec& Sp) {
    DevCtrl* C = P.ctrl;
    const unsigned listed = *Sp.nremovals;
    const unsigned n = listed < Sp.max_removals ? listed : Sp.max_removals;
    const unsigned ca = C->cur[Sp.A], cb = C->cur[Sp.B];
    for (unsigned r = threadIdx.x; r < n; r += blockDim.x) {
        P.sp[Sp.A].x[ca][Sp.removal[2 * r]] = dead_marker();
        P.sp[Sp.B].x[cb][Sp.removal[2 * r + 1]] = dead_marker();
    }
    pdl_trigger();
    if (threadIdx.x == 0 && n) {
        atomicAdd(&C->removed[Sp.A], (unsigned long long)n);
        atomicAdd(&C->removed[Sp.B], (unsigned long long)n);
        atomicAdd(Sp.reacted, (unsigned long long)n);
    }
}

// (22) e + O- -> O + 2e: the reacted pairs (O- slot, e slot), listed in any
// order by k_pair, in one block.  Each pair's kinematics continue the O-'s
// stream after its acceptance number: the share u of E_rel - E_th taken by
// the detached electron, then one isotropic direction for each electron; the
// electron keeps going from the O-'s velocity with the rest, the O- is marked
// dead (its charge was taken out by k_pair), and the newborn is staged at the
// rank of its O- parent's slot among the listed pairs (the method's order),
// its charge into the births' deposit.  The end-of-step kernel places the
// newborns after the step's other electron births.
__device__ __forceinline__ void edet_apply_body(const Params& P, const PairSpec& Sp) {
    __shared__ unsigned sh_wtries;
    DevCtrl* C = P.ctrl;
    if (threadIdx.x == 0) sh_wtries = 0u;
    __syncthreads();
    const unsigned listed = *Sp.nremovals;
    const unsigned n = listed < Sp.max_removals ? listed : Sp.max_removals;
    const unsigned long long step = C->step;
    const unsigned ca = C->cur[Sp.A], cb = C->cur[Sp.B];
    const SpeciesBuf& SA = P.sp[Sp.A];
    const SpeciesBuf& SB = P.sp[Sp.B];
    unsigned wtries = 0;
    for (unsigned r = threadIdx.x; r < n; r += blockDim.x) {
        const unsigned a = Sp.removal[2 * r], b = Sp.removal[2 * r + 1];
        unsigned rank = 0;   // slots of the O- are distinct: each reacts once
        for (unsigned q = 0; q < n; ++q) rank += (Sp.removal[2 * q] < a) ? 1u : 0u;
        const float ax = SA.x[ca][a], avx = SA.vx[ca][a], avy = SA.vy[ca][a], avz = SA.vz[ca][a];
        const uint32_t id = SA.id[ca][a];
        const float gx = avx - SB.vx[cb][b], gy = avy - SB.vy[cb][b], gz = avz - SB.vz[cb][b];
        const float E = Sp.kappa * dot3(gx, gy, gz, gx, gy, gz);
        const float Er = E - Sp.thr;
        Stream st;
        st.init(id, P.seed, step, Sp.tag_pair);
        (void)st.next();                         // the acceptance number
        const float us = uniform(st.next());
        const float Es = us * Er;
        const float Ep = Er - Es;
        float n1x, n1y, n1z, n2x, n2y, n2z;
        isotropic(st, n1x, n1y, n1z, wtries);
        isotropic(st, n2x, n2y, n2z, wtries);
        const float vp = sqrtf(Ep / P.kappa[SP_E]);
        const float vs = sqrtf(Es / P.kappa[SP_E]);
        SB.vx[cb][b] = avx + vp * n1x;
        SB.vy[cb][b] = avy + vp * n1y;
        SB.vz[cb][b] = avz + vp * n1z;
        SA.x[ca][a] = dead_marker();
        P.stage22[rank] = make_float4(ax, avx + vs * n2x, avy + vs * n2y, avz + vs * n2z);
        int j; float f;
        cell_of(ax, P.inv_dx, P.Nc, j, f);
        const uint32_t rr = cic_r(f);
        atomicAdd(&P.Qb[SP_E][j], (unsigned long long)(65536u - rr));
        if (rr) atomicAdd(&P.Qb[SP_E][j + 1], (unsigned long long)rr);
    }
    pdl_trigger();
    if (wtries) atomicAdd(&sh_wtries, wtries);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (n) {
            atomicAdd(&C->removed[Sp.A], (unsigned long long)n);
            atomicAdd(Sp.reacted, (unsigned long long)n);
        }
        C->births22 = n;
        if (sh_wtries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh_wtries);
    }
}

__global__ void __launch_bounds__(HIST_T) k_pair_hist(Params P, PairSpec Sp) {
    pdl_wait();
    pair_hist_body(P, Sp, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(PAIR_T) k_pair(Params P, PairSpec Sp) {
    pdl_wait();
    pair_body(P, Sp, blockIdx.x, gridDim.x);
}

// one block: the lists are short
__global__ void k_pair_apply(Params P, PairSpec Sp) {
    pdl_wait();
    pair_apply_body(P, Sp);
}

// batched: block b works for discharge map[b].x (block map[b].y of map[b].z)
__global__ void __launch_bounds__(HIST_T) k_pair_hist_b(const Params* __restrict__ all,
                                                         const PairSpec* __restrict__ specs,
                                                         const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    const uint4 m = map[blockIdx.x];
    const PairSpec Sp = specs[m.x];
    if (!Sp.active) return;   // block-uniform
    load_params(sP, all + m.x);
    pair_hist_body(sP, Sp, m.y, m.z);
}

__global__ void __launch_bounds__(PAIR_T) k_pair_b(const Params* __restrict__ all, const PairSpec* __restrict__ specs,
                                                    const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    const uint4 m = map[blockIdx.x];
    const PairSpec Sp = specs[m.x];
    if (!Sp.active) return;
    load_params(sP, all + m.x);
    pair_body(sP, Sp, m.y, m.z);
}

__global__ void k_edet_apply(Params P, PairSpec Sp) {
    pdl_wait();
    edet_apply_body(P, Sp);
}

// batched: block d applies discharge d's (22) list
__global__ void k_edet_apply_b(const Params* __restrict__ all, const PairSpec* __restrict__ specs) {
    __shared__ Params sP;
    pdl_wait();
    const PairSpec Sp = specs[blockIdx.x];
    if (!Sp.active) return;
    load_params(sP, all + blockIdx.x);
    edet_apply_body(sP, Sp);
}

// batched: block d applies discharge d's list
__global__ void k_pair_apply_b(const Params* __restrict__ all, const PairSpec* __restrict__ specs) {
    __shared__ Params sP;
    pdl_wait();
    const PairSpec Sp = specs[blockIdx.x];
    if (!Sp.active) return;
    load_params(sP, all + blockIdx.x);
    pair_apply_body(sP, Sp);
}

}  // namespace

size_t pair_hist_smem_bytes(int Nc) { return 3 * sizeof(unsigned) * (size_t)Nc; }

cudaError_t configure_pair_hist_smem(int Nc) {
    cudaError_t e = cudaFuncSetAttribute(k_pair_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pair_hist_smem_bytes(Nc));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_hist_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_hist_smem_bytes(Nc));
    return e;
}

void launch_pair_hist(const Params& P, const PairSpec& S, int grid, cudaStream_t s) {
    launch_pdl(k_pair_hist, grid, HIST_T, pair_hist_smem_bytes(P.Nc), s, P, S);
}

void launch_pair(const Params& P, const PairSpec& S, int grid, cudaStream_t s) {
    launch_pdl(k_pair, grid, PAIR_T, 0, s, P, S);
}

// the list counter is cleared by the end-of-step kernel
void launch_pair_apply(const Params& P, const PairSpec& S, cudaStream_t s) {
    launch_pdl(k_pair_apply, 1, 256, 0, s, P, S);
}

void launch_edet_apply(const Params& P, const PairSpec& S, cudaStream_t s) {
    launch_pdl(k_edet_apply, 1, 256, 0, s, P, S);
}

void launch_edet_apply_batched(const Params* all, const PairSpec* specs, int n, cudaStream_t s) {
    launch_pdl(k_edet_apply_b, n, 256, 0, s, all, specs);
}

void launch_pair_hist_batched(const Params* all, const PairSpec* specs, const uint4* map, int nblocks, size_t smem,
                              cudaStream_t s) {
    launch_pdl(k_pair_hist_b, nblocks, HIST_T, smem, s, all, specs, map);
}

void launch_pair_batched(const Params* all, const PairSpec* specs, const uint4* map, int nblocks, cudaStream_t s) {
    launch_pdl(k_pair_b, nblocks, PAIR_T, 0, s, all, specs, map);
}

void launch_pair_apply_batched(const Params* all, const PairSpec* specs, int n, cudaStream_t s) {
    launch_pdl(k_pair_apply_b, n, 256, 0, s, all, specs);
}

}  // namespace o2
