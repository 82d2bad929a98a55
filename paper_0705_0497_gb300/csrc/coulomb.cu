// Coulomb elastic collisions (1)-(6) of Table 1 (e-e, O- - O-, O2+ - O2+,
// e - O2+, e - O-, O- - O2+), by the binary collision model of Takizuka & Abe
// (J. Comput. Phys. 25, 205, 1977), on ion steps with dt_ion, after the
// species' pushes and collisions and before the reactive pairs (22), (16),
// (17); reactions in the order (1)..(6).
//
// Within a cell each pair's relative velocity u (|u| = g) turns by theta,
// tan(theta/2) = delta ~ N(0, sigma^2), sigma^2 = K N / g^3 with
// K = q_a^2 q_b^2 w lnL dt_ion / (8 pi eps0^2 mu^2 A dx), and an azimuth phi
// uniform on [0, 2 pi); the pair's momentum and energy are kept.  Pairs from
// the cell lists in array order: like species the rotated list (r a random
// shift per cell) in consecutive pairs (an odd one sits out), N = the
// species' count in the cell; unlike species the i-th of the shorter list
// with member (i + r) mod M of the longer, N = M.  delta from the first
// member's stream (tag 12 + reaction index): one polar normal, then phi as
// the double angle of a uniform point of the unit disk (no trigonometric
// function: the same rounding as the oracle's).
//
// GPU form: on a Coulomb step each species taking part is sorted by cell
// (stable: array order within a cell) in three passes over its tiles of
// TILE slots: per-tile cell counts, a scan of each cell's counts over the
// tiles (and of the cell totals), and a scatter that ranks the slots of a
// tile per cell warp by warp (each warp owns a contiguous chunk, its rounds
// of 32 in slot order, ranks within a round from __match_any_sync).  One
// kernel per reaction then runs the cell's pairs, a block per cell.
#include "common.cuh"

namespace o2 {

namespace {

constexpr int CT = 256;                       // threads of the count, scatter and pair kernels
constexpr int SCAN_T = 1024;                  // threads of the column scan (32 cells x 32 warps)
constexpr int CHUNK_W = TILE / (CT / 32);     // slots of a tile per scatter warp (1024)

// Per-tile cell counts of the live particles of species S: hist[tile][cell].
template <int S>
__global__ void __launch_bounds__(CT) k_cell_count(Params P) {
    extern __shared__ unsigned cnt[];         // [Nc]
    pdl_wait();
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const unsigned long long ns = C->slots[S] < P.sp[S].cap ? C->slots[S] : P.sp[S].cap;
    const unsigned ntiles = (unsigned)ceil_div(ns, TILE);
    const float* __restrict__ X = P.sp[S].x[C->cur[S]];
    unsigned* __restrict__ H = P.chist[S];
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int c = threadIdx.x; c < Nc; c += CT) cnt[c] = 0u;
        __syncthreads();
        const unsigned long long base = (unsigned long long)t * TILE;
        for (int k = threadIdx.x; k < TILE; k += CT) {
            const unsigned long long p = base + k;
            if (p < ns) {
                const float x = X[p];
                if (!is_dead(x)) {
                    int c; float f;
                    cell_of(x, P.inv_dx, Nc, c, f);
                    atomicAdd(&cnt[c], 1u);
                }
            }
        }
        __syncthreads();
        for (int c = threadIdx.x; c < Nc; c += CT) H[(size_t)t * Nc + c] = cnt[c];
        __syncthreads();
    }
    pdl_trigger();
}

// Each cell's counts over the tiles turned into offsets (exclusive scan
// along the tiles, in place), and the cell totals.  A block takes 32 cells
// (lane = cell), its 32 warps contiguous ranges of tiles.
template <int S>
__global__ void __launch_bounds__(SCAN_T) k_cell_colscan(Params P) {
    __shared__ unsigned part[32][33];
    pdl_wait();
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc;
    const unsigned long long ns = C->slots[S] < P.sp[S].cap ? C->slots[S] : P.sp[S].cap;
    const unsigned T = (unsigned)ceil_div(ns, TILE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const unsigned per = (T + 31) / 32;
    const unsigned t0 = warp * per < T ? warp * per : T, t1 = t0 + per < T ? t0 + per : T;
    unsigned* __restrict__ H = P.chist[S];
    unsigned sum = 0;
    if (c < Nc)
        for (unsigned t = t0; t < t1; ++t) sum += H[(size_t)t * Nc + c];
    part[warp][lane] = sum;
    __syncthreads();
    if (warp == 0) {
        unsigned run = 0;
        for (int w = 0; w < 32; ++w) { const unsigned v = part[w][lane]; part[w][lane] = run; run += v; }
        if (c < Nc) P.ctot[S][c] = run;
    }
    __syncthreads();
    if (c < Nc) {
        unsigned run = part[warp][lane];
        for (unsigned t = t0; t < t1; ++t) {
            const unsigned v = H[(size_t)t * Nc + c];
            H[(size_t)t * Nc + c] = run;
            run += v;
        }
    }
    pdl_trigger();
}

// Start of each cell's list: exclusive scan of the cell totals (one block).
template <int S>
__global__ void __launch_bounds__(SCAN_T) k_cell_start(Params P) {
    __shared__ unsigned ws[32];
    pdl_wait();
    const int Nc = P.Nc;
    const int per = (Nc + SCAN_T - 1) / SCAN_T;
    const int c0 = threadIdx.x * per;
    unsigned local = 0;
    for (int i = 0; i < per; ++i) if (c0 + i < Nc) local += P.ctot[S][c0 + i];
    unsigned total;
    unsigned run = block_excl_scan<SCAN_T>(local, ws, &total);
    for (int i = 0; i < per; ++i)
        if (c0 + i < Nc) { P.cstart[S][c0 + i] = run; run += P.ctot[S][c0 + i]; }
    pdl_trigger();
}

// Rows of the per-warp counts have an even length, so that the 32-bit
// shared-memory atomics on pairs of 16-bit counts stay 4-byte aligned.
__host__ __device__ inline int even(int n) { return (n + 1) & ~1; }

// Stable scatter of the slots of species S into cell order.
template <int S>
__global__ void __launch_bounds__(CT) k_cell_scatter(Params P) {
    extern __shared__ unsigned short wcnt[];  // [CT/32][even(Nc)]: per-warp counts, then offsets
    pdl_wait();
    DevCtrl* C = P.ctrl;
    const int Nc = P.Nc, NcE = even(P.Nc);
    const unsigned long long ns = C->slots[S] < P.sp[S].cap ? C->slots[S] : P.sp[S].cap;
    const unsigned ntiles = (unsigned)ceil_div(ns, TILE);
    const float* __restrict__ X = P.sp[S].x[C->cur[S]];
    const unsigned* __restrict__ H = P.chist[S];
    const unsigned* __restrict__ cst = P.cstart[S];
    unsigned* __restrict__ out = P.csort[S];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned short* mine = wcnt + warp * NcE;
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int k = threadIdx.x; k < (CT / 32) * NcE; k += CT) wcnt[k] = 0;
        __syncthreads();
        const unsigned long long base = (unsigned long long)t * TILE + (unsigned long long)warp * CHUNK_W;
        for (int r = 0; r < CHUNK_W; r += 32) {
            const unsigned long long p = base + r + lane;
            if (p < ns) {
                const float x = X[p];
                if (!is_dead(x)) {
                    int c; float f;
                    cell_of(x, P.inv_dx, Nc, c, f);
                    atomicAdd(reinterpret_cast<unsigned*>(&mine[c & ~1]), (c & 1) ? 0x10000u : 1u);
                }
            }
        }
        __syncthreads();
        // per cell: offsets of the warps' chunks within the tile
        for (int c = threadIdx.x; c < Nc; c += CT) {
            unsigned run = 0;
            for (int w = 0; w < CT / 32; ++w) {
                const unsigned v = wcnt[w * NcE + c];
                wcnt[w * NcE + c] = (unsigned short)run;
                run += v;
            }
        }
        __syncthreads();
        for (int r = 0; r < CHUNK_W; r += 32) {
            const unsigned long long p = base + r + lane;
            int c = -1;
            if (p < ns) {
                const float x = X[p];
                if (!is_dead(x)) { float f; cell_of(x, P.inv_dx, Nc, c, f); }
            }
            const unsigned peers = __match_any_sync(0xffffffffu, c);
            unsigned off = 0;
            if (c >= 0) off = mine[c];
            __syncwarp();
            if (c >= 0) {
                const unsigned rank = __popc(peers & lt);
                out[cst[c] + H[(size_t)t * Nc + c] + off + rank] = (unsigned)p;
                if (rank == 0) mine[c] = (unsigned short)(off + __popc(peers));
            }
            __syncwarp();
        }
        __syncthreads();
    }
    pdl_trigger();
}

// One pair of reaction r: particle ia of species a, ib of species b.
__device__ __forceinline__ void coulomb_pair(const Params& P, int r, int a, unsigned ia, int b, unsigned ib, float N,
                                             unsigned long long n, unsigned& wtries, unsigned& npairs) {
    DevCtrl* C = P.ctrl;
    const unsigned ca = C->cur[a], cb = C->cur[b];
    float* AX = P.sp[a].vx[ca]; float* AY = P.sp[a].vy[ca]; float* AZ = P.sp[a].vz[ca];
    float* BX = P.sp[b].vx[cb]; float* BY = P.sp[b].vy[cb]; float* BZ = P.sp[b].vz[cb];
    float ax = AX[ia], ay = AY[ia], az = AZ[ia];
    float bx = BX[ib], by = BY[ib], bz = BZ[ib];
    const float ux = ax - bx, uy = ay - by, uz = az - bz;
    const float g2 = dot3(ux, uy, uz, ux, uy, uz);
    if (!(g2 > 0.0f)) return;
    const float g = sqrtf(g2);
    Stream st;
    st.init(P.sp[a].id[ca][ia], P.seed, n, TAG_COUL + (uint32_t)r);
    float z0, z1;
    normal_pair(st, z0, z1, wtries);
    const float sig2 = P.coul_K[r] * N / (g2 * g);
    const float d = sqrtf(sig2) * z0;
    float sn, omc;
    if (fabsf(d) < 1e18f) {
        const float q = 1.0f / (1.0f + d * d);
        sn = 2.0f * d * q;
        omc = 2.0f * (d * d) * q;
    } else {
        sn = 0.0f; omc = 2.0f;
    }
    float cp = 1.0f, spn = 0.0f;
    for (int t = 0; t < MAX_TRIES; ++t) {
        const float e1 = 2.0f * uniform(st.next()) - 1.0f;
        const float e2 = 2.0f * uniform(st.next()) - 1.0f;
        const float s2 = e1 * e1 + e2 * e2;
        if (s2 > 0.0f && s2 < 1.0f) { cp = (e1 * e1 - e2 * e2) / s2; spn = (2.0f * e1 * e2) / s2; break; }
        if (t == MAX_TRIES - 1) ++wtries;
    }
    const float up2 = ux * ux + uy * uy;
    float dx, dy, dz;
    if (up2 > 0.0f) {
        const float up = sqrtf(up2);
        const float sc = sn * cp, ss = sn * spn;
        dx = (ux * uz / up) * sc - (uy * g / up) * ss - ux * omc;
        dy = (uy * uz / up) * sc + (ux * g / up) * ss - uy * omc;
        dz = -up * sc - uz * omc;
    } else {
        dx = g * (sn * cp);
        dy = g * (sn * spn);
        dz = -uz * omc;
    }
    const float fa = P.coul_fa[r], fb = P.coul_fb[r];
    AX[ia] = ax + fa * dx; AY[ia] = ay + fa * dy; AZ[ia] = az + fa * dz;
    BX[ib] = bx - fb * dx; BY[ib] = by - fb * dy; BZ[ib] = bz - fb * dz;
    ++npairs;
}

// Reaction r (species a, b): a block per cell (grid-stride), its pairs spread
// over the block's threads (disjoint particles: no two threads touch one).
__global__ void __launch_bounds__(CT) k_coulomb(Params P, int r, int a, int b) {
    __shared__ unsigned sh_shift, sh_tries, sh_pairs;
    pdl_wait();
    DevCtrl* C = P.ctrl;
    const unsigned long long n = C->step;
    const int Nc = P.Nc;
    if (threadIdx.x == 0) { sh_tries = 0u; sh_pairs = 0u; }
    unsigned wtries = 0, npairs = 0;
    for (int c = blockIdx.x; c < Nc; c += gridDim.x) {
        const unsigned na = P.ctot[a][c], nb = (a == b) ? na : P.ctot[b][c];
        if (a == b ? na < 2u : (na == 0u || nb == 0u)) continue;   // block-uniform
        const unsigned M = na > nb ? na : nb, m = na < nb ? na : nb;
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)n, TAG_SHIFT_COUL + (uint32_t)r, 0u, (uint32_t)(n >> 32)),
                                          make_uint2((uint32_t)c, P.seed));
            sh_shift = w.x % M;
        }
        __syncthreads();
        const unsigned rs = sh_shift;
        const unsigned* LA = P.csort[a] + P.cstart[a][c];
        const unsigned* LB = P.csort[b] + P.cstart[b][c];
        if (a == b) {
            for (unsigned j = threadIdx.x; 2u * j + 1u < na; j += CT) {
                const unsigned k1 = (unsigned)(((unsigned long long)rs + 2ull * j) % na);
                const unsigned k2 = (unsigned)(((unsigned long long)rs + 2ull * j + 1ull) % na);
                coulomb_pair(P, r, a, LA[k1], a, LA[k2], (float)na, n, wtries, npairs);
            }
        } else {
            const bool a_short = na <= nb;
            for (unsigned i = threadIdx.x; i < m; i += CT) {
                const unsigned q = (unsigned)(((unsigned long long)i + rs) % M);
                coulomb_pair(P, r, a, a_short ? LA[i] : LA[q], b, a_short ? LB[q] : LB[i], (float)M, n, wtries,
                             npairs);
            }
        }
    }
    pdl_trigger();
    if (wtries) atomicAdd(&sh_tries, wtries);
    if (npairs) atomicAdd(&sh_pairs, npairs);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sh_tries) atomicAdd(&C->cnt.warn_tries, (unsigned long long)sh_tries);
        if (sh_pairs) atomicAdd(&C->cnt.coulomb_pairs, (unsigned long long)sh_pairs);
    }
}

template <int S>
void sort_species(const Params& P, int grid, cudaStream_t s) {
    const int Nc = P.Nc;
    launch_pdl(k_cell_count<S>, grid, CT, sizeof(unsigned) * (size_t)Nc, s, P);
    launch_pdl(k_cell_colscan<S>, (Nc + 31) / 32, SCAN_T, 0, s, P);
    launch_pdl(k_cell_start<S>, 1, SCAN_T, 0, s, P);
    launch_pdl(k_cell_scatter<S>, grid, CT, sizeof(unsigned short) * (CT / 32) * (size_t)even(Nc), s, P);
}

}  // namespace

const int COUL_SPECIES[6][2] = {{SP_E, SP_E}, {SP_OM, SP_OM}, {SP_OP, SP_OP}, {SP_E, SP_OP}, {SP_E, SP_OM},
                                {SP_OM, SP_OP}};

cudaError_t configure_coulomb_smem(int Nc) {
    const int sc = (int)(sizeof(unsigned short) * (CT / 32) * (size_t)even(Nc));
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_scatter<SP_E>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_scatter<SP_OM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_scatter<SP_OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
    return e;
}

// The Coulomb collisions of one ion step (mask bit r-1 = reaction r): the
// species taking part sorted by cell, then the reactions in order.  Returns
// the number of kernels launched.
int launch_coulomb(const Params& P, unsigned mask, int grid, cudaStream_t s) {
    int launches = 0;
    unsigned need = 0;
    for (int r = 0; r < 6; ++r)
        if ((mask >> r) & 1u) need |= (1u << COUL_SPECIES[r][0]) | (1u << COUL_SPECIES[r][1]);
    if (need & 1u) { sort_species<SP_E>(P, grid, s); launches += 4; }
    if (need & 2u) { sort_species<SP_OM>(P, grid, s); launches += 4; }
    if (need & 4u) { sort_species<SP_OP>(P, grid, s); launches += 4; }
    const int cgrid = P.Nc < 4096 ? P.Nc : 4096;
    for (int r = 0; r < 6; ++r) {
        if (!((mask >> r) & 1u)) continue;
        launch_pdl(k_coulomb, cgrid, CT, 0, s, P, r, COUL_SPECIES[r][0], COUL_SPECIES[r][1]);
        ++launches;
    }
    return launches;
}

}  // namespace o2
