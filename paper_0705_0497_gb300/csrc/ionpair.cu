// Ion-ion neutralization (17), O- + O2+ -> O + O2, on ion steps: a binary,
// cell-local (DSMC-like) process at the post-push positions.
//
// Pairing (the reading used by the oracle): in cell c take the surviving O-
// and O2+ in array order, n- and n+ of them, m = min, M = max, and a shift
// r_c drawn per cell and step; the i-th member of the shorter list (O- on a
// tie), i < m, is paired with member (i + r_c) mod M of the longer one.  A
// pair reacts with probability P = M w sigma_n(E_rel) g dt_ion / (A dx).
//
// GPU form: k_pair_hist counts, per 8192-slot tile, the surviving ions per
// cell of both species.  k_pair_scan turns these into
// per-cell exclusive prefixes over tiles (so the rank of an ion in its cell
// list is prefix + its rank inside the tile) and draws the shifts.  k_pair
// gives each block one O- tile, split among its warps; with per-warp cell
// counts every O- learns its rank k in its cell list, whether it is paired
// and the rank q of its partner.  The acceptance
// draw needs only the O- id; since P <= K_max M w dt/(A dx), only the rare
// draws below that bound need the partner, which the warp then finds by a
// binary search over the O2+ prefixes and a ballot scan of one O2+ tile.
#include "common.cuh"

namespace o2 {

namespace {

constexpr int SCAN_T = 1024;   // 32 cells x 32 tile groups
constexpr int HIST_T = 512;

// Per 8192-slot tile of each ion species, the number of live ions per cell
// (post-push positions): hist[sp][tile][cell].  Blocks take tiles of O-
// first, then of O2+.
__global__ void __launch_bounds__(HIST_T) k_pair_hist(Params P) {
    extern __shared__ unsigned hsm[];
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const unsigned long long nsm = C->slots[SP_OM], nsp = C->slots[SP_OP];
    const unsigned ntm = (unsigned)ceil_div(nsm, TILE), ntp = (unsigned)ceil_div(nsp, TILE);
    for (unsigned g = blockIdx.x; g < ntm + ntp; g += gridDim.x) {
        const int sp = (g < ntm) ? 0 : 1;
        const unsigned tile = (g < ntm) ? g : g - ntm;
        const int S = sp == 0 ? SP_OM : SP_OP;
        const unsigned long long n = sp == 0 ? nsm : nsp;
        const float* X = P.sp[S].x[C->cur[S]];
        for (int c = threadIdx.x; c < Nc; c += HIST_T) hsm[c] = 0u;
        __syncthreads();
        const unsigned long long base = (unsigned long long)tile * TILE;
        const unsigned long long end = (base + TILE < n) ? base + TILE : n;
#pragma unroll 4
        for (unsigned long long i = base + threadIdx.x; i < end; i += HIST_T) {
            const float x = X[i];
            if (!is_dead(x)) {
                int c; float fr;
                cell_of(x, P.inv_dx, Nc, c, fr);
                atomicAdd(&hsm[c], 1u);
            }
        }
        __syncthreads();
        unsigned* H = P.hist[sp] + (size_t)tile * Nc;
        for (int c = threadIdx.x; c < Nc; c += HIST_T) H[c] = hsm[c];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_T) k_pair_scan(Params P) {
    __shared__ unsigned part[32][33];
    __shared__ unsigned tot[2][32];
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const int cl = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cl;
    for (int sp = 0; sp < 2; ++sp) {
        const unsigned long long ns = C->slots[sp == 0 ? SP_OM : SP_OP];
        const unsigned ntiles = (unsigned)ceil_div(ns, TILE);
        const unsigned per = (ntiles + 31) / 32;
        const unsigned t0 = g * per, t1 = (t0 + per < ntiles) ? t0 + per : ntiles;
        unsigned* H = P.hist[sp];
        unsigned sum = 0;
        if (c < Nc)
            for (unsigned t = t0; t < t1; ++t) sum += H[(size_t)t * Nc + c];
        part[g][cl] = sum;
        __syncthreads();
        unsigned before = 0;
        for (int k = 0; k < g; ++k) before += part[k][cl];
        if (g == 31) tot[sp][cl] = before + sum;
        __syncthreads();
        if (c < Nc) {
            unsigned run = before;
            for (unsigned t = t0; t < t1; ++t) {
                const unsigned v = H[(size_t)t * Nc + c];
                H[(size_t)t * Nc + c] = run;
                run += v;
            }
        }
        __syncthreads();
    }
    if (g == 0 && c < Nc) {
        const unsigned nm = tot[0][cl], npl = tot[1][cl];
        const unsigned m = nm < npl ? nm : npl, M = nm < npl ? npl : nm;
        unsigned r = 0;
        if (m > 0) {
            const unsigned long long step = C->step;
            const uint4 w = philox4x32_10(make_uint4((uint32_t)step, TAG_SHIFT, 0u, (uint32_t)(step >> 32)),
                                          make_uint2((uint32_t)c, P.seed));
            r = w.x % M;
            atomicAdd(&C->cnt.pair_candidates, (unsigned long long)m);
        }
        P.cellinfo[4 * c + 0] = nm;
        P.cellinfo[4 * c + 1] = npl;
        P.cellinfo[4 * c + 2] = r;
    }
}

constexpr int PAIR_WARPS = 8;

// Slot of the O2+ with rank q in cell c (cell list in slot order).
__device__ unsigned find_op(const Params& P, const float* XP, unsigned long long nsl, unsigned ntiles, int c,
                            unsigned q, int lane) {
    const int Nc = P.Nc;
    const unsigned* H = P.hist[1];
    // largest tile t with prefix(t, c) <= q
    unsigned lo = 0, hi = ntiles;   // answer in [lo, hi)
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (H[(size_t)mid * Nc + c] <= q) lo = mid; else hi = mid;
    }
    const unsigned want = q - H[(size_t)lo * Nc + c];
    const unsigned long long base = (unsigned long long)lo * TILE;
    const unsigned long long end = (base + TILE < nsl) ? base + TILE : nsl;
    unsigned seen = 0;
    for (unsigned long long b = base; b < end; b += 32) {
        const unsigned long long p = b + lane;
        bool hit = false;
        if (p < end) {
            const float x = XP[p];
            if (!is_dead(x)) {
                int j; float fr;
                cell_of(x, P.inv_dx, Nc, j, fr);
                hit = (j == c);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const unsigned cnt = __popc(bal);
        if (seen + cnt > want) {
            // the (want - seen)-th set bit
            unsigned bits = bal;
            for (unsigned k = 0; k < want - seen; ++k) bits &= bits - 1;
            return (unsigned)(b + (__ffs(bits) - 1));
        }
        seen += cnt;
    }
    return 0xFFFFFFFFu;
}

// One block per O- tile.  Pass 1: each warp loads its sub-range of the tile
// (all loads in flight together), stores each slot's cell (or "dead") in
// shared memory and counts its ions per cell.  Pass 2: per cell, prefix of
// the warps' counts, starting from the tile's prefix over earlier tiles.
// Pass 3: each warp walks its sub-range in slot order from shared memory;
// an O- learns its rank k in its cell list, whether it is paired, and draws
// its acceptance number; the rare candidates find their partner.
__global__ void __launch_bounds__(PAIR_WARPS * 32) k_pair(Params P, int W) {
    extern __shared__ unsigned pair_smem[];
    unsigned short* cell16 = reinterpret_cast<unsigned short*>(pair_smem);   // [TILE]
    unsigned* whist = pair_smem + TILE / 2;                                  // [W][Nc]
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long step = C->step;
    const unsigned long long nsm = C->slots[SP_OM], nsp = C->slots[SP_OP];
    const unsigned ntm = (unsigned)ceil_div(nsm, TILE), ntp = (unsigned)ceil_div(nsp, TILE);
    const unsigned cm = C->cur[SP_OM], cp = C->cur[SP_OP];
    const float* XM = P.sp[SP_OM].x[cm];
    const uint32_t* IDM = P.sp[SP_OM].id[cm];
    const float* XP = P.sp[SP_OP].x[cp];
    const float pf = P.pair_factor;
    const int sub = TILE / W;
    unsigned gt1 = 0;
    unsigned* myhist = whist + (size_t)warp * Nc;

    for (unsigned tile = blockIdx.x; tile < ntm; tile += gridDim.x) {
        for (int i = threadIdx.x; i < W * Nc; i += blockDim.x) whist[i] = 0u;
        __syncthreads();
        const unsigned long long base = (unsigned long long)tile * TILE;
        const unsigned long long end = (base + TILE < nsm) ? base + TILE : nsm;
        const unsigned long long s0 = base + (unsigned long long)warp * sub;
        const unsigned long long s1 = (s0 + sub < end) ? s0 + sub : end;
        // pass 1
#pragma unroll 4
        for (unsigned long long b = s0; b < s1; b += 32) {
            const unsigned long long p = b + lane;
            if (p < s1) {
                const float x = XM[p];
                unsigned short cc = 0xFFFFu;
                if (!is_dead(x)) {
                    int c; float fr;
                    cell_of(x, P.inv_dx, Nc, c, fr);
                    cc = (unsigned short)c;
                    atomicAdd(&myhist[c], 1u);
                }
                cell16[p - base] = cc;
            }
        }
        __syncthreads();
        // pass 2
        const unsigned* HM = P.hist[0] + (size_t)tile * Nc;
        for (int c = threadIdx.x; c < Nc; c += blockDim.x) {
            unsigned run = HM[c];
            for (int w = 0; w < W; ++w) {
                const unsigned v = whist[(size_t)w * Nc + c];
                whist[(size_t)w * Nc + c] = run;
                run += v;
            }
        }
        __syncthreads();
        // pass 3
        for (unsigned long long b = s0; b < s1; b += 32) {
            const unsigned long long p = b + lane;
            int c = 0;
            bool live = false;
            if (p < s1) {
                const unsigned short cc = cell16[p - base];
                if (cc != 0xFFFFu) { live = true; c = cc; }
            }
            const unsigned lmask = __ballot_sync(0xffffffffu, live);
            bool cand = false;
            unsigned q = 0, M = 0;
            float u = 0.0f;
            if (live) {
                const unsigned peers = __match_any_sync(lmask, c);
                const unsigned lt = peers & ((1u << lane) - 1u);
                const unsigned before = myhist[c];
                const unsigned k = before + __popc(lt);
                __syncwarp(lmask);
                if (lt == 0u) myhist[c] = before + __popc(peers);
                const unsigned nm = P.cellinfo[4 * c], npl = P.cellinfo[4 * c + 1], r = P.cellinfo[4 * c + 2];
                const unsigned m = nm < npl ? nm : npl;
                M = nm < npl ? npl : nm;
                bool paired = false;
                if (m > 0) {
                    if (nm <= npl) { q = (unsigned)(((unsigned long long)k + r) % M); paired = true; }
                    else {
                        const unsigned i = (unsigned)(((unsigned long long)k + M - r) % M);
                        if (i < m) { q = i; paired = true; }
                    }
                }
                if (paired) {
                    const uint4 w = philox4x32_10(make_uint4((uint32_t)step, TAG_PAIR, 0u, (uint32_t)(step >> 32)),
                                                  make_uint2(IDM[p], P.seed));
                    u = uniform(w.x);
                    cand = u < P.Kmax_hi * (pf * (float)M);
                }
            }
            __syncwarp();
            unsigned cmask = __ballot_sync(0xffffffffu, cand);
            while (cmask) {
                const int owner = __ffs(cmask) - 1;
                cmask &= cmask - 1;
                const int oc = __shfl_sync(0xffffffffu, c, owner);
                const unsigned oq = __shfl_sync(0xffffffffu, q, owner);
                const unsigned b_slot = find_op(P, XP, nsp, ntp, oc, oq, lane);
                if (lane == owner && b_slot != 0xFFFFFFFFu) {
                    const SpeciesBuf& SM = P.sp[SP_OM];
                    const SpeciesBuf& SPp = P.sp[SP_OP];
                    const float gx = SM.vx[cm][p] - SPp.vx[cp][b_slot];
                    const float gy = SM.vy[cm][p] - SPp.vy[cp][b_slot];
                    const float gz = SM.vz[cm][p] - SPp.vz[cp][b_slot];
                    const float E = P.kappa_n * dot3(gx, gy, gz, gx, gy, gz);
                    int gi; float gw; bool above;
                    grid_locate(E, gi, gw, above);
                    if (above) atomicAdd(&C->cnt.warn_emax, 1ull);
                    const float K = grid_interp(P.Ktab, 1, 0, gi, gw);
                    const float Pp = K * (pf * (float)M);
                    if (Pp > 1.0f) ++gt1;
                    if (u < Pp) {
                        const unsigned idx = atomicAdd(&C->removals, 1u);
                        if (idx < P.max_removals) {
                            P.removal[2 * idx] = (unsigned)p;
                            P.removal[2 * idx + 1] = b_slot;
                        }
                        // take both out of the fresh deposit
                        int j; float f;
                        cell_of(XM[p], P.inv_dx, Nc, j, f);
                        uint32_t rr = cic_r(f);
                        atomicAdd(&P.Qf[SP_OM][j], 0ull - (unsigned long long)(65536u - rr));
                        atomicAdd(&P.Qf[SP_OM][j + 1], 0ull - (unsigned long long)rr);
                        cell_of(XP[b_slot], P.inv_dx, Nc, j, f);
                        rr = cic_r(f);
                        atomicAdd(&P.Qf[SP_OP][j], 0ull - (unsigned long long)(65536u - rr));
                        atomicAdd(&P.Qf[SP_OP][j + 1], 0ull - (unsigned long long)rr);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (gt1) atomicAdd(&C->cnt.warn_pair_gt1, (unsigned long long)gt1);
}

}  // namespace

void launch_pair_hist(const Params& P, int grid, cudaStream_t s) {
    k_pair_hist<<<grid, HIST_T, sizeof(unsigned) * (size_t)P.Nc, s>>>(P);
}

void launch_pair_scan(const Params& P, cudaStream_t s) {
    k_pair_scan<<<(P.Nc + 31) / 32, SCAN_T, 0, s>>>(P);
}

// warps per block: the largest of 8, 4, 2, 1 whose per-warp cell counts fit
int pair_warps(int Nc) {
    for (int w = PAIR_WARPS; w > 1; w >>= 1)
        if (2 * TILE + 4 * (size_t)w * Nc <= 200 * 1024) return w;
    return 1;
}

size_t pair_smem_bytes(int Nc) {
    return 2 * (size_t)TILE + 4 * (size_t)pair_warps(Nc) * Nc;
}

void launch_pair(const Params& P, int grid, cudaStream_t s) {
    const int W = pair_warps(P.Nc);
    k_pair<<<grid, W * 32, pair_smem_bytes(P.Nc), s>>>(P, W);
}

cudaError_t configure_pair_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace o2
