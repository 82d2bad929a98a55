// Shared definitions of the o2pic CUDA library (host runtime + kernels).
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "o2pic.h"

namespace o2 {

// Programmatic stream serialization is on except while a graph with one
// branch per discharge is captured: there, the early-launched blocks of many
// branches could hold pieces of every SM while single-block kernels of other
// branches wait for a whole one.
extern thread_local bool pdl_enabled;

// Launch with programmatic stream serialization (see pdl_wait in common.cuh).
template <typename... Params_, typename... Args>
inline void launch_pdl(void (*kernel)(Params_...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


constexpr int NSP = 3;
constexpr int SP_E = 0, SP_OM = 1, SP_OP = 2;
constexpr int MAXPROC = O2PIC_MAXPROC;

// Rate-table grid: 32 points per octave on [2^-10, 2^12] eV (705 points).
constexpr int GRID_SUB_BITS = 5;
constexpr int NGRID = 22 * 32 + 1;
constexpr unsigned GRID_BASE = (127u - 10u) << GRID_SUB_BITS;   // (bits >> 18) at 2^-10
constexpr float GRID_EMIN = 0.0009765625f;                       // 2^-10
constexpr float GRID_EMAX = 4096.0f;                             // 2^12

constexpr int BLOCK = 256;              // threads of the particle kernels
constexpr int ITEMS = 4;                // particles per thread per chunk (one float4)
constexpr int CHUNK = BLOCK * ITEMS;    // 1024
constexpr int TILE = 8192;              // slots per tile (compaction, neutralization histograms)
constexpr int WTILE = 2048;             // slots per warp work unit of the particle kernels
constexpr int CHUNKS_PER_TILE = TILE / CHUNK;
constexpr int FLUSH_TILES = 7;          // tiles between deposit flushes (7*8192*2^16 < 2^32)
constexpr int MAX_TRIES = 32;           // rejection-loop cap
constexpr uint32_t FIX_ONE = 65536u;    // CIC fixed point per particle
constexpr int QCAP = BLOCK - 1 + CHUNK; // candidate queue capacity
constexpr int MAX_NODES = 8193;         // grid limit (smem field and histograms)
constexpr int JRING = 8192;             // steps of conduction-current sums kept on the device
// Copies of a species' fresh deposit Qf (Ng each): the particle kernel's
// blocks flush their cell histograms into copy (block mod QCOPIES), so the
// 64-bit reductions of one step spread over QCOPIES times more L2 lines; the
// end-of-step kernel sums the copies (integers: the sum is exact).  Other
// deposits into Qf use copy 0.
constexpr int QCOPIES = 4;

enum Kind { K_ELASTIC = 0, K_EXCITE = 1, K_IONIZE = 2, K_ATTACH = 3, K_DETACH = 4, K_CX = 5, K_NEUTRALIZE = 6 };
// TAG_FLIGHT + s: the first free-flight draw of a particle of species s (at a
// load or at its birth).
enum Tag : uint32_t { TAG_E = 0, TAG_OM = 1, TAG_OP = 2, TAG_PAIR = 3, TAG_SHIFT = 4, TAG_REC = 5, TAG_SHIFT_REC = 6,
                      TAG_FLIGHT = 7, TAG_EDET = 10, TAG_SHIFT_EDET = 11, TAG_COUL = 12, TAG_SHIFT_COUL = 18 };

// device error bits
constexpr unsigned long long ERR_CAPACITY = 1ull, ERR_ID = 2ull, ERR_NONFINITE = 4ull, ERR_TIMEOUT = 8ull;

// kernel kinds (timing, tickets)
enum KernelKind { KK_PUSH_E = 0, KK_PUSH_OM = 1, KK_PUSH_OP = 2, KK_PAIR_HIST = 3, KK_PAIR = 4,
                  KK_FIELD = 5, KK_COMPACT = 6, KK_DEPOSIT = 7, KK_CAND_E = 8, KK_CAND_OM = 9, KK_CAND_OP = 10,
                  KK_REC = 11, KK_FILT_OM = 12, KK_FILT_OP = 13, KK_COUL = 14, NKK = 15 };

// Counters: same layout as the head of o2pic_stats.
struct DevCounters {
    unsigned long long events[NSP][MAXPROC];
    unsigned long long absorbed[NSP][2];
    unsigned long long born[NSP];
    unsigned long long neutralized, pair_candidates, particle_steps;
    unsigned long long warn_emax, warn_tries, warn_pair_gt1;
    unsigned long long id_overflow;
    unsigned long long psteps[NSP];
    unsigned long long recombined, rec_candidates;
    unsigned long long edetached, edet_candidates;
    unsigned long long coulomb_pairs;
    unsigned long long warn_numax;
};

// Births appended by one kernel into species d: births of the electron
// kernel (e from ionization, O2+ from ionization, O- from attachment) and of
// the O- kernel (e from detachment) in that canonical order.
enum BirthSlot { B_E_FROM_E = 0, B_OP_FROM_E = 1, B_OM_FROM_E = 2, B_E_FROM_OM = 3, NB = 4 };

// Device-resident step state; read by every kernel, committed by the field kernel.
struct DevCtrl {
    unsigned long long step;               // current step n
    unsigned long long field_step;         // the same, kept by the field-solve block
    unsigned long long epoch;              // distinct per step, never reused (look-back flags)
    unsigned long long slots[NSP];         // array slots in use (live + dead) before this step's births
    unsigned long long live[NSP];
    unsigned long long removed[NSP];       // removed this step (absorbed, consumed, neutralized)
    unsigned long long births[NB];         // this step's births per BirthSlot
    unsigned long long acc_steps;          // steps summed into Qacc
    unsigned long long error_flags;
    unsigned long long next_id[NSP];       // id of the next birth (ids above 2^32 - 1 overflow)
    unsigned int cur[NSP];                 // current buffer (ping-pong) per species
    unsigned int ticket[NKK + NSP];        // tile tickets per kernel kind, + compaction per species
    unsigned int removals;                 // (17) pairs to remove
    unsigned int rremovals;                // (16) pairs to remove
    unsigned int dremovals;                // (22) pairs listed
    unsigned int births22;                 // (22) electron births staged this step
    DevCounters cnt;
};

// tc: the step of each particle's next collision candidate (the end of its
// current free flight), low 32 bits of the step index.
struct SpeciesBuf {
    float* x[2];
    float* vx[2];
    float* vy[2];
    float* vz[2];
    uint32_t* id[2];
    uint32_t* tc[2];
    unsigned long long cap;
};

// Everything the kernels need; passed by value.
struct Params {
    DevCtrl* ctrl;
    SpeciesBuf sp[NSP];
    // rate tables (cumulative, FP32), [NGRID][nproc]
    const float* cum[NSP];
    int nproc[NSP];
    int kind[NSP][MAXPROC];
    float thr[NSP][MAXPROC];
    float numax[NSP], pmax[NSP];
    // free flights: species s is pushed every sub[s] steps; a gap of K pushes
    // is floor(ln(u) inv_lnq[s]) with inv_lnq = 1 / ln(1 - P_max) = -1 /
    // (nu_max dt_s), capped at kcap[s] (2^30 steps ahead, beyond any run)
    float inv_lnq[NSP], kcap[NSP];
    unsigned sub[NSP];
    int births_possible[NSP];
    int cum_smem[NSP];           // particle kernel stages the cumulative table in shared memory
    // (17)
    const float* Ktab;           // [NGRID] sigma_n g
    float Kmax_hi;               // max(Ktab) inflated so the prefilter bounds every interpolant
    int have_neutral;
    // grid / field
    int Nc, Ng;
    float inv_dx, Lf;
    double dx, c_field, U, two_pi_f, dt;   // c_field = e w dx / (A eps0 2^16)
    double inv_dx64, inv_2dx64;            // 1/dx and 1/(2 dx)
    double inv_Nc64;                       // 1/Nc when Nc is a power of two (exact), else 0
    const double* vring;         // electrode voltage U sin(2 pi f t_k) at t_k = k dt, slot k & vring_mask
    unsigned int vring_mask;
    float* Ef;                   // [Ng] gather field (FP32)
    double* phi;                 // [Ng], evaluated on request from fS, fU, fVD
    long long* fS;               // [Ng] S_j of the last field solve (exact prefix sums)
    long long* fU;               // [Ng] U_j of the last field solve
    double* fVD;                 // [2] V0, D0 of the last field solve
    unsigned long long* jring;   // [JRING][NSP] conduction-current sums (int64 mod 2^64), slot = step % JRING
    unsigned long long* Q[NSP];  // committed node charge
    unsigned long long* Qf[NSP]; // fresh deposit of the species pushed this step, QCOPIES x Ng
    unsigned long long* Qb[NSP]; // deposit of this step's births
    unsigned long long* Qacc[NSP];
    // per-species constants (FP32, computed once on the host)
    float dt_s[NSP], qmdt[NSP], kappa[NSP], a_m[NSP], a_M[NSP], sig_birth[NSP];
    float delta_el, sig_gas, kappa_n, pair_factor;
    uint32_t seed;
    // decoupled look-back state: per kernel kind, flag and value words per tile
    unsigned long long* lb_flag[NKK];
    unsigned long long* lb_val[NKK];
    unsigned int max_tiles;
    // births staging, [wtile * WTILE + rank] per BirthSlot, and the number
    // staged by each warp work unit (B_OP_FROM_E shares B_E_FROM_E's counts)
    float4* stage[NB];
    unsigned int* wcount[NB];
    unsigned int push_warps[NSP];  // warps of each particle kernel launch (units of wcount)
    // collision records at each particle warp's range, two uint4 each:
    // electrons {slot, id, x, vx}{vy, vz, -, -} per real collision; ions
    // {slot, id, vx, vy}{vz, w1, w2, w3} per candidate, compacted to the
    // real ones by the filter
    uint4* cand[NSP];
    unsigned int* ccount[NSP];     // records per warp
    unsigned int max_push_warps;   // bound on push_warps (shared memory of the field kernel)
    // (17): per-tile per-cell counts of live ions [2][max_tiles][Nc], per-cell info
    unsigned int* hist[2];       // 0: O-, 1: O2+
    unsigned int* ptot;          // [2][Nc]: live O-, O2+ per cell (cleared by the end-of-step kernel)
    unsigned int* removal;       // [2 * max_removals]: O- slot, O2+ slot
    unsigned int max_removals;
    // (16): per-tile per-cell counts of live e and O2+, per-cell totals, pairs
    const float* Ktab_r;         // [NGRID] sigma_r g
    float Kmax_r_hi, kappa_r;
    int have_recomb;
    unsigned int* rhist[2];      // 0: e, 1: O2+
    unsigned int* rtot;          // [2][Nc] (cleared by the end-of-step kernel)
    unsigned int* rremoval;      // [2 * max_rremovals]: e slot, O2+ slot
    unsigned int max_rremovals;
    // (22): per-tile per-cell counts of live O- and e, per-cell totals, pairs,
    // and the staged electron births in the order of their O- parents
    const float* Ktab_d;         // [NGRID] sigma_22 g
    float Kmax_d_hi, kappa_d, thr_d;
    int have_edet;
    unsigned int* dhist[2];      // 0: O-, 1: e
    unsigned int* dtot;          // [2][Nc] (cleared by the end-of-step kernel)
    unsigned int* dremoval;      // [2 * max_dremovals]: O- slot, e slot
    unsigned int max_dremovals;
    float4* stage22;             // [max_dremovals]
    // Coulomb (1)-(6): enabled reactions (bit r-1), per reaction the sigma^2
    // factor K and the shares m_b/(m_a+m_b), m_a/(m_a+m_b) of the change of
    // u; per species the cell sort of a Coulomb step: slots in cell order,
    // per-tile cell offsets, cell totals and cell starts
    unsigned int coul_mask;
    float coul_K[6], coul_fa[6], coul_fb[6];
    unsigned int* csort[NSP];
    unsigned int* chist[NSP];
    unsigned int* ctot[NSP];
    unsigned int* cstart[NSP];
    // compaction trigger
    float compact_dead_frac;
};

// A cell-binned binary process between species A and B (the reading of
// (17), also used for (16)): A's id draws the acceptance number; reacted
// pairs go to a removal list (A slot, B slot).
struct PairSpec {
    int A, B;
    unsigned int* histA;         // [tiles of A][Nc] live A per cell
    unsigned int* histB;
    unsigned int* tot;           // [2][Nc]: A, B per cell
    const float* K;              // [NGRID] sigma g
    float Kmax_hi, kappa;
    uint32_t tag_pair, tag_shift;
    unsigned int* removal;
    unsigned int* nremovals;     // device counter of listed pairs
    unsigned int max_removals;
    unsigned long long* tested;  // device counter of pairs tested
    unsigned long long* reacted; // device counter of pairs removed (the apply kernel's)
    int active;                  // 0: the discharge has no such process (batched launches skip it)
    float thr;                   // a pair reacts only at or above this relative energy [eV]
    int b_survives;              // 1: only A is removed (B's charge stays), (22)
};

__host__ __device__ inline unsigned long long ceil_div(unsigned long long a, unsigned long long b) {
    return (a + b - 1) / b;
}

// The particle kernels give warp w of W warps the contiguous slot range
// [w R, min((w+1) R, n)) with R = this length (128-aligned).
__host__ __device__ inline unsigned warp_range_len(unsigned n, unsigned W) {
    const unsigned per = (n + W - 1) / W;
    return ((per + 127u) / 128u) * 128u;
}

// ---------------------------------------------------------------- launchers
// (defined in the kernel translation units, called by the runtime)
void launch_push(int species, const Params& P, int grid, cudaStream_t s);
void launch_cand(int species, const Params& P, int grid, cudaStream_t s);   // ion species
// true when the ion filter and kinematics run inside the ion particle kernels
// (then the filter and kinematics kernels are not launched)
bool ions_fused();
// true when the particle kernel may stage the cumulative rate table in shared
// memory (it does when the table keeps its resident blocks per SM)
bool cum_smem_allowed();
void launch_filter(int species, const Params& P, int grid, cudaStream_t s);
void launch_filter_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s);
void launch_pair_hist(const Params& P, const PairSpec& S, int grid, cudaStream_t s);
cudaError_t configure_pair_hist_smem(int Nc);
void launch_pair(const Params& P, const PairSpec& S, int grid, cudaStream_t s);
void launch_pair_apply(const Params& P, const PairSpec& S, cudaStream_t s);
void launch_edet_apply(const Params& P, const PairSpec& S, cudaStream_t s);
int launch_coulomb(const Params& P, unsigned mask, int grid, cudaStream_t s);
cudaError_t configure_coulomb_smem(int Nc);
void launch_edet_apply_batched(const Params* all, const PairSpec* specs, int n, cudaStream_t s);
// batched launches (one grid for many discharges; map[b] = discharge, block, blocks)
void launch_push_batched(int species, const Params* all, const uint4* map, int nblocks, size_t smem, cudaStream_t s);
void launch_cand_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s);
void launch_field_batched(const Params* all, int n, size_t smem, int mode, int pushed_mask, cudaStream_t s);
void launch_compact_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s);
void launch_pair_hist_batched(const Params* all, const PairSpec* specs, const uint4* map, int nblocks, size_t smem,
                              cudaStream_t s);
void launch_pair_batched(const Params* all, const PairSpec* specs, const uint4* map, int nblocks, cudaStream_t s);
void launch_pair_apply_batched(const Params* all, const PairSpec* specs, int n, cudaStream_t s);
void launch_field(const Params& P, int mode, int pushed_mask, cudaStream_t s);
void launch_phi(const Params& P, cudaStream_t s);
void launch_compact(int species, const Params& P, int grid, cudaStream_t s);
void launch_deposit(int species, const Params& P, int grid, cudaStream_t s);
void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, unsigned long long n, cudaStream_t s);
void launch_ln(const float* x, float* out, unsigned long long n, cudaStream_t s);
void launch_load_check(int species, const Params& P, unsigned long long n, cudaStream_t s);
void launch_gather(int species, const Params& P, int grid, unsigned long long epoch, unsigned* ticket,
                   unsigned long long* flag, unsigned long long* val, float* x, float* vx, float* vy, float* vz,
                   uint32_t* id, uint32_t* tc, unsigned long long cap, unsigned long long* out_count, cudaStream_t s);
void launch_flight_init(int species, const Params& P, cudaStream_t s);
cudaError_t configure_push_smem(size_t max_bytes);
cudaError_t configure_field_smem(size_t bytes);
size_t field_smem_bytes(const Params& P);
int push_occupancy(int species, const Params& P, int* blocks_per_sm);
size_t push_smem_bytes(int species, const Params& P);

}  // namespace o2
