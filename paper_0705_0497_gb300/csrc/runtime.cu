// Host runtime and C ABI of libo2pic (include/o2pic.h): context and device
// memory, rate-table construction, particle loading, the per-step launch
// sequence, readback, timing and error reporting.
//
// The rate tables follow the null-collision method of the paper's Sec. 2:
// per species s and process k, nu_k(E_i) = n_target sigma_k(E_i) g(E_i) on the
// 705-point grid (32 per octave over [2^-10, 2^12] eV), g = sqrt(2 e E / mu),
// mu = m_e for electrons (target at rest) and the reduced mass for ions;
// cumulative sums in process order, nu_max = their maximum over the grid and
// P_max = 1 - exp(-nu_max dt_s).  Built in FP64, stored in FP32.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace o2 {
thread_local bool pdl_enabled = true;

// Ion chains on their own streams on ion steps (1), or all on the step's
// stream (0); programmatic dependent launches inside the graph of a batch of
// one discharge (1), or only outside graphs (0).  Both keep the results.  On
// the 512-cell, 1.6e7-particle discharge at its periodic state the fork took
// the RF cycle from 46.2 to 44.3 ms; the programmatic launches inside the
// one-discharge graph gained nothing (46.7 ms without the fork, 44.1 with).
#ifndef O2PIC_ION_FORK
#define O2PIC_ION_FORK 1
#endif
#ifndef O2PIC_GRAPH_PDL_SINGLE
#define O2PIC_GRAPH_PDL_SINGLE 0
#endif
constexpr bool ION_FORK = O2PIC_ION_FORK != 0;
}

// particle kernels run at most this many blocks per SM (bounds the per-warp
// birth counts the field kernel scans in shared memory)
constexpr int MAX_PUSH_BLOCKS_PER_SM = 8;

// The particle kernel keeps its shared-memory deposit as (count << 40) + sum
// of CIC weights per cell, so one block may deposit fewer than 2^24 particles
// into one cell.  A block handles at most slots / blocks + 8 * 128 slots, so
// at least capacity / 2^23 blocks per species keep it below 2^24 with margin.
int min_push_blocks(unsigned long long cap) {
    return (int)std::max<unsigned long long>(1, o2::ceil_div(cap, 1ull << 23));
}

using namespace o2;

namespace {

// CODATA 2018 (SI)
const double QE = 1.602176634e-19;
const double KB = 1.380649e-23;
const double EPS0 = 8.8541878128e-12;
const double TWO_PI = 6.283185307179586476925286766559;

struct HostProc {
    int kind, target;
    double thr;
    std::vector<double> E, s;
};

double grid_energy(int i) {
    return std::ldexp(1.0 + (i % 32) / 32.0, i / 32 - 10);
}

double sigma_at(const HostProc& p, double E) {
    if (E < p.thr) return 0.0;
    const size_t n = p.E.size();
    if (E <= p.E[0]) return p.s[0];
    if (E >= p.E[n - 1]) return p.s[n - 1];
    const size_t b = std::upper_bound(p.E.begin(), p.E.end(), E) - p.E.begin();
    const double Ea = p.E[b - 1], Eb = p.E[b], sa = p.s[b - 1], sb = p.s[b];
    return sa + (sb - sa) * ((E - Ea) / (Eb - Ea));
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

}  // namespace

struct o2pic_ctx {
    o2pic_config cfg;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t last = nullptr;
    // ion steps: the O- and O2+ chains on their own streams beside the
    // electron kernel (forked from and joined back into the step's stream)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    Params P;
    DevCtrl* d_ctrl = nullptr;
    std::vector<void*> allocs;
    // host state
    unsigned long long host_step = 0;
    unsigned since_check = 0;
    bool dirty = true;
    bool have_tables = false;
    bool loaded[NSP] = {false, false, false};
    bool flight_ok[NSP] = {false, false, false};   // free flights known (else drawn by prepare)
    double ecap[NSP] = {INFINITY, INFINITY, INFINITY};   // majorant caps (eV) of the next set_processes
    bool coul_alloc = false;                       // Coulomb cell-sort buffers allocated
    int latched = 0;
    int grid_push[NSP] = {0, 0, 0};
    int grid_pair = 0, grid_pair_e = 0, grid_compact = 0, grid_deposit = 0;
    unsigned long long launches = 0;
    unsigned long long gen = 0;        // bumped by every call that invalidates a captured graph
    unsigned long long ring_start = 0; // first step recorded in the current-sum ring
    // gather (read_particles) state
    unsigned* d_gticket = nullptr;
    unsigned long long* d_gflag = nullptr;
    unsigned long long* d_gval = nullptr;
    unsigned long long* d_gcount = nullptr;
    unsigned long long gepoch = 0;
    // electrode-voltage ring (device) and the highest step index filled
    double* d_vring = nullptr;
    // timing
    bool timing = false;
    struct Ev { cudaEvent_t a, b; int kind; };
    std::vector<Ev> pending;
    std::vector<cudaEvent_t> pool;
    double ms[NKK] = {0};
    unsigned long long nlaunch[NKK] = {0};
};

namespace {

int cuda_fail(o2pic_ctx* c, cudaError_t e) {
    if (e == cudaSuccess) return O2PIC_OK;
    if (c) c->latched = c->latched ? c->latched : O2PIC_E_CUDA;
    return O2PIC_E_CUDA;
}

template <class T>
cudaError_t ctx_alloc(o2pic_ctx* c, T** p, size_t count) {
    cudaError_t e = dalloc(p, count);
    if (e == cudaSuccess) {
        c->allocs.push_back((void*)*p);
        e = cudaMemset(*p, 0, sizeof(T) * (count ? count : 1));
    }
    return e;
}

cudaStream_t pick(o2pic_ctx* c, void* s) {
    cudaStream_t st = s ? (cudaStream_t)s : c->stream;
    c->last = st;
    return st;
}

cudaEvent_t take_event(o2pic_ctx* c) {
    if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void harvest_timing(o2pic_ctx* c) {
    for (auto& ev : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev.a, ev.b) == cudaSuccess) c->ms[ev.kind] += t;
        c->pool.push_back(ev.a);
        c->pool.push_back(ev.b);
    }
    c->pending.clear();
}

// Launch wrapper: optional event pair around the launch.
template <class F>
void launch(o2pic_ctx* c, int kind, cudaStream_t s, F&& f) {
    if (c->timing) {
        if (c->pending.size() >= 8192) { cudaStreamSynchronize(s); harvest_timing(c); }
        o2pic_ctx::Ev ev{take_event(c), take_event(c), kind};
        cudaEventRecord(ev.a, s);
        f();
        cudaEventRecord(ev.b, s);
        c->pending.push_back(ev);
    } else {
        f();
    }
    c->nlaunch[kind] += 1;
    c->launches += 1;
}

int check_flags(o2pic_ctx* c) {
    unsigned long long flags = 0;
    cudaError_t e = cudaMemcpy(&flags, &c->d_ctrl->error_flags, sizeof(flags), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    int code = O2PIC_OK;
    if (flags & ERR_CAPACITY) code = O2PIC_E_CAPACITY;
    else if (flags & ERR_ID) code = O2PIC_E_ID_OVERFLOW;
    else if (flags & ERR_NONFINITE) code = O2PIC_E_NONFINITE;
    else if (flags & ERR_TIMEOUT) code = O2PIC_E_TIMEOUT;
    if (code && !c->latched) c->latched = code;
    return c->latched;
}

int sync_all(o2pic_ctx* c) {
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (c->timing) harvest_timing(c);
    return check_flags(c);
}

int validate(const o2pic_config* g) {
    if (!g) return O2PIC_E_INVALID_ARG;
    if (!(g->L > 0) || !(g->dt > 0) || !(g->f >= 0) || !(g->p >= 0) || !(g->T_gas > 0) || !(g->weight >= 0) ||
        !(g->area > 0) || !(g->C_meta >= 0) || !std::isfinite(g->U))
        return O2PIC_E_INVALID_ARG;
    if (!(g->m_e > 0) || !(g->m_OM > 0) || !(g->m_OP > 0) || !(g->M_gas > 0)) return O2PIC_E_INVALID_ARG;
    if (g->n_cells < 1 || g->n_cells + 1 > MAX_NODES || g->ion_subcycle < 1) return O2PIC_E_INVALID_ARG;
    for (int s = 0; s < NSP; ++s)
        if (g->capacity[s] > (1ull << 31)) return O2PIC_E_INVALID_ARG;
    return O2PIC_OK;
}

void set_constants(o2pic_ctx* c) {
    const o2pic_config& g = c->cfg;
    Params& P = c->P;
    const double mass[NSP] = {g.m_e, g.m_OM, g.m_OP};
    const int charge[NSP] = {-1, -1, +1};
    const double dx = g.L / g.n_cells;
    for (int s = 0; s < NSP; ++s) {
        const double dts = g.dt * (s == SP_E ? 1.0 : (double)g.ion_subcycle);
        P.dt_s[s] = (float)dts;
        P.qmdt[s] = (float)((charge[s] * QE / mass[s]) * dts);
        const double mu = (s == SP_E) ? mass[s] : mass[s] * g.M_gas / (mass[s] + g.M_gas);
        P.kappa[s] = (float)(0.5 * mu / QE);
        P.a_m[s] = (float)(mass[s] / (mass[s] + g.M_gas));
        P.a_M[s] = (float)(g.M_gas / (mass[s] + g.M_gas));
        P.sig_birth[s] = (float)std::sqrt(KB * g.T_gas / mass[s]);
        P.sub[s] = (s == SP_E) ? 1u : (unsigned)g.ion_subcycle;
        P.inv_lnq[s] = -INFINITY;
        P.kcap[s] = (float)std::floor(1073741824.0 / (double)P.sub[s]);
    }
    P.delta_el = (float)(2.0 * g.m_e / g.M_gas);
    P.sig_gas = (float)std::sqrt(KB * g.T_gas / g.M_gas);
    P.inv_dx = (float)(1.0 / dx);
    P.Lf = (float)g.L;
    const double mun = g.m_OM * g.m_OP / (g.m_OM + g.m_OP);
    P.kappa_n = (float)(0.5 * mun / QE);
    const double mur = g.m_e * g.m_OP / (g.m_e + g.m_OP);
    P.kappa_r = (float)(0.5 * mur / QE);
    const double mud = g.m_e * g.m_OM / (g.m_e + g.m_OM);
    P.kappa_d = (float)(0.5 * mud / QE);
    const double dt_ion = g.dt * (double)g.ion_subcycle;
    P.pair_factor = (float)(g.weight * dt_ion / (g.area * dx));
    P.seed = g.seed;
    P.Nc = g.n_cells;
    P.Ng = g.n_cells + 1;
    P.dx = dx;
    P.c_field = QE * g.weight * dx / (g.area * EPS0 * 65536.0);
    P.inv_dx64 = 1.0 / dx;
    P.inv_2dx64 = 1.0 / (2.0 * dx);
    // x / Nc and x * (1 / Nc) are the same IEEE result when 1 / Nc is exact
    P.inv_Nc64 = (g.n_cells & (g.n_cells - 1)) == 0 ? 1.0 / (double)g.n_cells : 0.0;
    P.U = g.U;
    P.two_pi_f = TWO_PI * g.f;
    P.dt = g.dt;
    P.compact_dead_frac = 1.0f / 16.0f;
}

constexpr unsigned VRING = 4096;

// U sin(2 pi f t_k), t_k = k dt, for k in [k0, k1], into the device ring.
int fill_vring(o2pic_ctx* c, unsigned long long k0, unsigned long long k1, cudaStream_t s) {
    std::vector<double> v;
    v.reserve((size_t)(k1 - k0 + 1));
    for (unsigned long long k = k0; k <= k1; ++k) {
        const double t = (double)k * c->cfg.dt;
        v.push_back(c->cfg.U * std::sin(TWO_PI * c->cfg.f * t));
    }
    size_t i = 0;
    while (i < v.size()) {
        const unsigned slot = (unsigned)((k0 + i) & (VRING - 1));
        const size_t n = std::min<size_t>(v.size() - i, VRING - slot);
        cudaError_t e = cudaMemcpyAsync(c->d_vring + slot, v.data() + i, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(c, e);
        i += n;
    }
    return O2PIC_OK;
}

int prepare(o2pic_ctx* c, cudaStream_t s) {
    if (int rc = fill_vring(c, c->host_step, c->host_step, s)) return rc;
    Params& P = c->P;
    for (int sp = 0; sp < NSP; ++sp) {
        cudaMemsetAsync(P.Qf[sp], 0, sizeof(unsigned long long) * QCOPIES * P.Ng, s);
        cudaMemsetAsync(P.Qb[sp], 0, sizeof(unsigned long long) * P.Ng, s);
    }
    for (int sp = 0; sp < NSP; ++sp)
        launch(c, KK_DEPOSIT, s, [&] { launch_deposit(sp, P, c->grid_deposit, s); });
    // free flights of particles whose flights are not known, drawn at this step
    for (int sp = 0; sp < NSP; ++sp)
        if (!c->flight_ok[sp]) {
            launch_flight_init(sp, P, s);
            c->launches += 1;
            c->flight_ok[sp] = true;
        }
    launch(c, KK_FIELD, s, [&] { launch_field(P, 1, 7, s); });
    c->ring_start = c->host_step;
    c->dirty = false;
    return cuda_fail(c, cudaGetLastError());
}

// The cell-binned binary processes of a context: (22) e + O- -> O + 2e
// (A = O-, only A removed), (16) e + O2+ -> O + O, (17) O- + O2+ -> O + O2.
PairSpec spec_edet(o2pic_ctx* c) {
    const Params& P = c->P;
    return PairSpec{SP_OM, SP_E, P.dhist[0], P.dhist[1], P.dtot, P.Ktab_d, P.Kmax_d_hi, P.kappa_d, TAG_EDET,
                    TAG_SHIFT_EDET, P.dremoval, &c->d_ctrl->dremovals, P.max_dremovals,
                    &c->d_ctrl->cnt.edet_candidates, &c->d_ctrl->cnt.edetached, P.have_edet, P.thr_d, 1};
}
PairSpec spec_rec(o2pic_ctx* c) {
    const Params& P = c->P;
    return PairSpec{SP_E, SP_OP, P.rhist[0], P.rhist[1], P.rtot, P.Ktab_r, P.Kmax_r_hi, P.kappa_r, TAG_REC,
                    TAG_SHIFT_REC, P.rremoval, &c->d_ctrl->rremovals, P.max_rremovals,
                    &c->d_ctrl->cnt.rec_candidates, &c->d_ctrl->cnt.recombined, P.have_recomb, 0.0f, 0};
}
PairSpec spec_neu(o2pic_ctx* c) {
    const Params& P = c->P;
    return PairSpec{SP_OM, SP_OP, P.hist[0], P.hist[1], P.ptot, P.Ktab, P.Kmax_hi, P.kappa_n, TAG_PAIR,
                    TAG_SHIFT, P.removal, &c->d_ctrl->removals, P.max_removals,
                    &c->d_ctrl->cnt.pair_candidates, &c->d_ctrl->cnt.neutralized, P.have_neutral, 0.0f, 0};
}

// The kernel sequence of nsteps time steps on stream s (the electrode
// voltages of those steps must be in the ring already): electrons every step,
// ions and (17) on ion steps, the end-of-step kernel, and every compact_check
// steps a compaction check per species.  Host state advances with it.
void enqueue_steps(o2pic_ctx* c, uint64_t nsteps, cudaStream_t s) {
    Params& P = c->P;
    const unsigned S = (unsigned)c->cfg.ion_subcycle;
    for (uint64_t k = 0; k < nsteps; ++k) {
        const bool ion = (c->host_step % S) == 0;
        // on ion steps the three species' particle chains share nothing but
        // order-free atomics until the pair processes, so (unless the launches
        // are being timed one by one) the ion chains run on their own streams
        const bool fork = ion && ION_FORK && !c->timing;
        const cudaStream_t so = fork ? c->aux[0] : s, sp2 = fork ? c->aux[1] : s;
        if (fork) {
            cudaEventRecord(c->ev_fork, s);
            cudaStreamWaitEvent(so, c->ev_fork, 0);
            cudaStreamWaitEvent(sp2, c->ev_fork, 0);
        }
        launch(c, KK_PUSH_E, s, [&] { launch_push(SP_E, P, c->grid_push[SP_E], s); });
        if (ion) {
            launch(c, KK_PUSH_OM, so, [&] { launch_push(SP_OM, P, c->grid_push[SP_OM], so); });
            if (P.nproc[SP_OM] && !ions_fused()) {
                launch(c, KK_FILT_OM, so, [&] { launch_filter(SP_OM, P, c->grid_push[SP_OM], so); });
                launch(c, KK_CAND_OM, so, [&] { launch_cand(SP_OM, P, c->grid_push[SP_OM], so); });
            }
            launch(c, KK_PUSH_OP, sp2, [&] { launch_push(SP_OP, P, c->grid_push[SP_OP], sp2); });
            if (P.nproc[SP_OP] && !ions_fused()) {
                launch(c, KK_FILT_OP, sp2, [&] { launch_filter(SP_OP, P, c->grid_push[SP_OP], sp2); });
                launch(c, KK_CAND_OP, sp2, [&] { launch_cand(SP_OP, P, c->grid_push[SP_OP], sp2); });
            }
            if (fork) {
                cudaEventRecord(c->ev_join[0], so);
                cudaEventRecord(c->ev_join[1], sp2);
                cudaStreamWaitEvent(s, c->ev_join[0], 0);
                cudaStreamWaitEvent(s, c->ev_join[1], 0);
            }
            if (P.coul_mask) {
                int k = 0;
                launch(c, KK_COUL, s, [&] { k = launch_coulomb(P, P.coul_mask, c->grid_compact, s); });
                c->launches += (unsigned long long)(k - 1);
            }
            if (P.have_edet) {
                const PairSpec D = spec_edet(c);
                launch(c, KK_REC, s, [&] { launch_pair_hist(P, D, c->grid_compact, s); });
                launch(c, KK_REC, s, [&] { launch_pair(P, D, c->grid_pair, s); });
                launch(c, KK_REC, s, [&] { launch_edet_apply(P, D, s); });
            }
            if (P.have_recomb) {
                const PairSpec R = spec_rec(c);
                launch(c, KK_REC, s, [&] { launch_pair_hist(P, R, c->grid_compact, s); });
                launch(c, KK_REC, s, [&] { launch_pair(P, R, c->grid_pair_e, s); });
                launch(c, KK_REC, s, [&] { launch_pair_apply(P, R, s); });
            }
            if (P.have_neutral) {
                const PairSpec N = spec_neu(c);
                launch(c, KK_PAIR_HIST, s, [&] { launch_pair_hist(P, N, c->grid_compact, s); });
                launch(c, KK_PAIR, s, [&] { launch_pair(P, N, c->grid_pair, s); });
            }
        }
        launch(c, KK_FIELD, s, [&] { launch_field(P, 0, ion ? 7 : 1, s); });
        c->host_step += 1;
        if (++c->since_check >= c->cfg.compact_check) {
            for (int sp = 0; sp < NSP; ++sp)
                launch(c, KK_COMPACT, s, [&] { launch_compact(sp, P, c->grid_compact, s); });
            c->since_check = 0;
        }
    }
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

int o2pic_version(void) { return 1; }

const char* o2pic_strerror(int code) {
    switch (code) {
    case O2PIC_OK: return "ok";
    case O2PIC_E_INVALID_ARG: return "invalid argument";
    case O2PIC_E_CAPACITY: return "particle capacity exceeded";
    case O2PIC_E_ID_OVERFLOW: return "particle id overflow (2^32)";
    case O2PIC_E_NONFINITE: return "non-finite or out-of-range particle";
    case O2PIC_E_CUDA: return "CUDA error";
    case O2PIC_E_TIMEOUT: return "bounded device wait gave up";
    case O2PIC_E_STATE: return "call out of order (tables or particles missing)";
    default: return "unknown error";
    }
}

int o2pic_config_init(o2pic_config* g) {
    if (!g) return O2PIC_E_INVALID_ARG;
    std::memset(g, 0, sizeof(*g));
    const double amu = 1.66053906660e-27;
    g->L = 0.02; g->f = 13.56e6; g->U = 200.0; g->p = 10.0; g->T_gas = 300.0; g->C_meta = 0.0;
    g->dt = 1.0 / (13.56e6 * 400.0); g->weight = 2.0e9; g->area = 1.0;
    g->m_e = 9.1093837015e-31; g->m_OM = 16.0 * amu; g->m_OP = 32.0 * amu; g->M_gas = 32.0 * amu;
    g->n_cells = 128; g->ion_subcycle = 1; g->seed = 0; g->compact_check = 16;
    return O2PIC_OK;
}

int o2pic_create(const o2pic_config* cfg, o2pic_ctx** out) {
    if (!out) return O2PIC_E_INVALID_ARG;
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    o2pic_ctx* c = new (std::nothrow) o2pic_ctx();
    if (!c) return O2PIC_E_CUDA;
    c->cfg = *cfg;
    if (c->cfg.compact_check == 0) c->cfg.compact_check = 16;
    c->device = cfg->device;
    std::memset(&c->P, 0, sizeof(Params));
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (int i = 0; i < 2; ++i) {
            if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
            if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
        }
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        for (int i = 0; i < 2; ++i) {
        if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return O2PIC_E_CUDA;
    }
    c->last = c->stream;
    set_constants(c);
    Params& P = c->P;
    const int Ng = P.Ng, Nc = P.Nc;
    unsigned long long maxcap = 0;
    for (int s = 0; s < NSP; ++s) maxcap = std::max<unsigned long long>(maxcap, cfg->capacity[s]);
    const unsigned long long max_tiles = ceil_div(maxcap, TILE) + 1;
    P.max_tiles = (unsigned)max_tiles;
#define TRY(x) do { e = (x); if (e != cudaSuccess) { o2pic_destroy(c); return O2PIC_E_CUDA; } } while (0)
    TRY(ctx_alloc(c, &c->d_ctrl, 1));
    P.ctrl = c->d_ctrl;
    for (int s = 0; s < NSP; ++s) {
        const unsigned long long cap = ((cfg->capacity[s] + 63) / 64) * 64;
        P.sp[s].cap = cfg->capacity[s];
        for (int b = 0; b < 2; ++b) {
            TRY(ctx_alloc(c, &P.sp[s].x[b], cap));
            TRY(ctx_alloc(c, &P.sp[s].vx[b], cap));
            TRY(ctx_alloc(c, &P.sp[s].vy[b], cap));
            TRY(ctx_alloc(c, &P.sp[s].vz[b], cap));
            TRY(ctx_alloc(c, &P.sp[s].id[b], cap));
            TRY(ctx_alloc(c, &P.sp[s].tc[b], cap));
        }
        float* cum;
        TRY(ctx_alloc(c, &cum, (size_t)NGRID * MAXPROC));
        P.cum[s] = cum;
        TRY(ctx_alloc(c, &P.Q[s], Ng));
        TRY(ctx_alloc(c, &P.Qf[s], (size_t)QCOPIES * Ng));
        TRY(ctx_alloc(c, &P.Qb[s], Ng));
        TRY(ctx_alloc(c, &P.Qacc[s], Ng));
    }
    float* K;
    TRY(ctx_alloc(c, &K, NGRID));
    P.Ktab = K;
    float* Kr;
    TRY(ctx_alloc(c, &Kr, NGRID));
    P.Ktab_r = Kr;
    TRY(ctx_alloc(c, &c->d_vring, VRING));
    P.vring = c->d_vring;
    P.vring_mask = VRING - 1;
    TRY(ctx_alloc(c, &P.Ef, Ng));
    TRY(ctx_alloc(c, &P.phi, Ng));
    TRY(ctx_alloc(c, &P.fS, Ng));
    TRY(ctx_alloc(c, &P.fU, Ng));
    TRY(ctx_alloc(c, &P.fVD, 2));
    TRY(ctx_alloc(c, &P.jring, (size_t)JRING * NSP));
    for (int k = 0; k < NKK; ++k) {
        TRY(ctx_alloc(c, &P.lb_flag[k], max_tiles));
        TRY(ctx_alloc(c, &P.lb_val[k], 2 * max_tiles));
    }
    const unsigned long long units_e = ceil_div(cfg->capacity[SP_E], WTILE) + 1;
    const unsigned long long units_om = ceil_div(cfg->capacity[SP_OM], WTILE) + 1;
    TRY(ctx_alloc(c, &P.stage[B_E_FROM_E], units_e * WTILE));
    TRY(ctx_alloc(c, &P.stage[B_OP_FROM_E], units_e * WTILE));
    TRY(ctx_alloc(c, &P.stage[B_OM_FROM_E], units_e * WTILE));
    TRY(ctx_alloc(c, &P.stage[B_E_FROM_OM], units_om * WTILE));
    const size_t max_warps = (size_t)c->num_sms * MAX_PUSH_BLOCKS_PER_SM * (BLOCK / 32);
    P.max_push_warps = (unsigned)max_warps;
    TRY(ctx_alloc(c, &P.wcount[B_E_FROM_E], max_warps));
    P.wcount[B_OP_FROM_E] = P.wcount[B_E_FROM_E];
    TRY(ctx_alloc(c, &P.wcount[B_OM_FROM_E], max_warps));
    TRY(ctx_alloc(c, &P.wcount[B_E_FROM_OM], max_warps));
    for (int s = 0; s < NSP; ++s) {
        TRY(ctx_alloc(c, &P.cand[s], 2 * (cfg->capacity[s] + 128)));
        TRY(ctx_alloc(c, &P.ccount[s], max_warps));
    }
    const unsigned long long tiles_ion = std::max(ceil_div(cfg->capacity[SP_OM], TILE), ceil_div(cfg->capacity[SP_OP], TILE)) + 1;
    TRY(ctx_alloc(c, &P.hist[0], tiles_ion * Nc));
    TRY(ctx_alloc(c, &P.hist[1], tiles_ion * Nc));
    // (16): e and O2+ tiles, totals, pair list
    TRY(ctx_alloc(c, &P.rhist[0], (ceil_div(cfg->capacity[SP_E], TILE) + 1) * Nc));
    TRY(ctx_alloc(c, &P.rhist[1], (ceil_div(cfg->capacity[SP_OP], TILE) + 1) * Nc));
    TRY(ctx_alloc(c, &P.rtot, 2 * (size_t)Nc));
    P.max_rremovals = (unsigned)std::max<unsigned long long>(1, std::min(cfg->capacity[SP_E], cfg->capacity[SP_OP]));
    TRY(ctx_alloc(c, &P.rremoval, 2 * (size_t)P.max_rremovals));
    TRY(ctx_alloc(c, &P.ptot, 2 * (size_t)Nc));
    // (22): O- and e tiles, totals, pair list, staged births
    float* Kd;
    TRY(ctx_alloc(c, &Kd, NGRID));
    P.Ktab_d = Kd;
    TRY(ctx_alloc(c, &P.dhist[0], (ceil_div(cfg->capacity[SP_OM], TILE) + 1) * Nc));
    TRY(ctx_alloc(c, &P.dhist[1], (ceil_div(cfg->capacity[SP_E], TILE) + 1) * Nc));
    TRY(ctx_alloc(c, &P.dtot, 2 * (size_t)Nc));
    P.max_dremovals = (unsigned)std::max<unsigned long long>(1, std::min(cfg->capacity[SP_OM], cfg->capacity[SP_E]));
    TRY(ctx_alloc(c, &P.dremoval, 2 * (size_t)P.max_dremovals));
    TRY(ctx_alloc(c, &P.stage22, (size_t)P.max_dremovals));
    P.max_removals = (unsigned)std::max<unsigned long long>(1, std::min(cfg->capacity[SP_OM], cfg->capacity[SP_OP]));
    TRY(ctx_alloc(c, &P.removal, 2 * (size_t)P.max_removals));
    TRY(ctx_alloc(c, &c->d_gticket, 1));
    TRY(ctx_alloc(c, &c->d_gflag, max_tiles));
    TRY(ctx_alloc(c, &c->d_gval, 2 * max_tiles));
    TRY(ctx_alloc(c, &c->d_gcount, 1));
    // kernel shared-memory opt-in and launch shapes
    size_t smax = 0;
    for (int s = 0; s < NSP; ++s) {
        P.nproc[s] = MAXPROC;
        P.cum_smem[s] = 1;
        smax = std::max(smax, push_smem_bytes(s, P));
    }
    smax = std::max(smax, sizeof(unsigned) * (size_t)Ng);
    TRY(configure_push_smem(smax));
    TRY(configure_field_smem(field_smem_bytes(P)));
    TRY(configure_pair_hist_smem(Nc));
    for (int s = 0; s < NSP; ++s) { P.nproc[s] = 0; P.cum_smem[s] = 0; }
    c->grid_pair = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(tiles_ion, 8ull * c->num_sms));
    c->grid_pair_e = (int)std::max<unsigned long long>(
        1, std::min<unsigned long long>(ceil_div(cfg->capacity[SP_E], TILE) + 1, 8ull * c->num_sms));
    c->grid_compact = 4 * c->num_sms;
    c->grid_deposit = 4 * c->num_sms;
    // steady initial control state
    DevCtrl h;
    std::memset(&h, 0, sizeof(h));
    h.epoch = 1;
    TRY(cudaMemcpy(c->d_ctrl, &h, sizeof(h), cudaMemcpyHostToDevice));
    TRY(cudaDeviceSynchronize());
#undef TRY
    *out = c;
    return O2PIC_OK;
}

void o2pic_destroy(o2pic_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (void* p : c->allocs) cudaFree(p);
    for (auto& ev : c->pending) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int o2pic_set_processes(o2pic_ctx* c, const o2pic_process* procs, int nproc) {
    if (!c || (nproc > 0 && !procs) || nproc < 0) return O2PIC_E_INVALID_ARG;
    const o2pic_config& g = c->cfg;
    std::vector<HostProc> sp[NSP];
    HostProc neutral, recomb, edet;
    bool have_neutral = false, have_recomb = false, have_edet = false;
    for (int j = 0; j < nproc; ++j) {
        const o2pic_process& q = procs[j];
        if (q.n < 1 || q.species < 0 || q.species >= NSP || !q.E_eV || !q.sigma_m2) return O2PIC_E_INVALID_ARG;
        if (q.kind < O2PIC_ELASTIC || q.kind > O2PIC_EDETACH) return O2PIC_E_INVALID_ARG;
        HostProc p;
        p.kind = q.kind; p.target = q.target; p.thr = q.threshold_eV;
        p.E.assign(q.E_eV, q.E_eV + q.n);
        p.s.assign(q.sigma_m2, q.sigma_m2 + q.n);
        for (int i = 1; i < q.n; ++i) if (!(p.E[i] > p.E[i - 1])) return O2PIC_E_INVALID_ARG;
        for (int i = 0; i < q.n; ++i) if (!(p.s[i] >= 0) || !std::isfinite(p.s[i])) return O2PIC_E_INVALID_ARG;
        if (q.kind == O2PIC_NEUTRALIZE) {
            if (have_neutral) return O2PIC_E_INVALID_ARG;
            neutral = p; have_neutral = true; continue;
        }
        if (q.kind == O2PIC_RECOMBINE) {
            if (have_recomb || q.species != SP_E) return O2PIC_E_INVALID_ARG;
            recomb = p; have_recomb = true; continue;
        }
        if (q.kind == O2PIC_EDETACH) {
            if (have_edet || q.species != SP_OM || !(q.threshold_eV >= 0)) return O2PIC_E_INVALID_ARG;
            edet = p; have_edet = true; continue;
        }
        // kinematics exist for: e: elastic, excite, ionize, attach; O-: elastic, detach; O2+: elastic, cx
        const bool ok = (q.species == SP_E && (q.kind == O2PIC_ELASTIC || q.kind == O2PIC_EXCITE ||
                                                q.kind == O2PIC_IONIZE || q.kind == O2PIC_ATTACH)) ||
                        (q.species == SP_OM && (q.kind == O2PIC_ELASTIC || q.kind == O2PIC_DETACH)) ||
                        (q.species == SP_OP && (q.kind == O2PIC_ELASTIC || q.kind == O2PIC_CX));
        if (!ok) return O2PIC_E_INVALID_ARG;
        if ((int)sp[q.species].size() >= MAXPROC) return O2PIC_E_INVALID_ARG;
        sp[q.species].push_back(p);
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e);
    Params& P = c->P;
    const double nO2 = g.p / (KB * g.T_gas);
    const double nmeta = g.C_meta * nO2;
    const double mass[NSP] = {g.m_e, g.m_OM, g.m_OP};
    for (int s = 0; s < NSP; ++s) {
        const int np = (int)sp[s].size();
        std::vector<float> cum((size_t)NGRID * std::max(np, 1), 0.0f);
        const double mu = (s == SP_E) ? mass[s] : mass[s] * g.M_gas / (mass[s] + g.M_gas);
        // nu_max over the grid points up to the first one at or above the
        // species' majorant cap (the whole grid without one): the linear
        // interpolant below the cap stays below it
        double mx = 0.0;
        bool capped = false;
        for (int i = 0; i < NGRID; ++i) {
            const double Ei = grid_energy(i);
            const double gv = std::sqrt(2.0 * QE * Ei / mu);
            double acc = 0.0;
            for (int k = 0; k < np; ++k) {
                const HostProc& pr = sp[s][k];
                const double ntar = (pr.target == O2PIC_TARGET_O2_META) ? nmeta : nO2;
                const double nu = ntar * sigma_at(pr, Ei) * gv;
                acc += nu;
                cum[(size_t)i * np + k] = (float)acc;
            }
            if (!capped) mx = std::max(mx, acc);
            if (Ei >= c->ecap[s]) capped = true;
        }
        const double dts = g.dt * (s == SP_E ? 1.0 : (double)g.ion_subcycle);
        P.nproc[s] = np;
        P.numax[s] = (float)mx;
        P.pmax[s] = (float)(1.0 - std::exp(-mx * dts));
        // 1 / ln(1 - P_max) for the free-flight draw; -inf when nu_max = 0
        P.inv_lnq[s] = (float)(-1.0 / (mx * dts));
        c->flight_ok[s] = false;   // flights drawn with the old nu_max: draw afresh
        bool births = false;
        for (int k = 0; k < np; ++k) {
            P.kind[s][k] = sp[s][k].kind;
            P.thr[s][k] = (float)sp[s][k].thr;
            if (sp[s][k].kind == O2PIC_IONIZE || sp[s][k].kind == O2PIC_ATTACH || sp[s][k].kind == O2PIC_DETACH)
                births = true;
        }
        P.births_possible[s] = births ? 1 : 0;
        if (np > 0) {
            e = cudaMemcpy((void*)P.cum[s], cum.data(), sizeof(float) * cum.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(c, e);
        }
    }
    std::vector<float> K(NGRID, 0.0f);
    float kmax = 0.0f;
    if (have_neutral) {
        const double mun = g.m_OM * g.m_OP / (g.m_OM + g.m_OP);
        for (int i = 0; i < NGRID; ++i) {
            const double Ei = grid_energy(i);
            const double gv = std::sqrt(2.0 * QE * Ei / mun);
            K[i] = (float)(sigma_at(neutral, Ei) * gv);
            kmax = std::max(kmax, K[i]);
        }
    }
    P.have_neutral = have_neutral ? 1 : 0;
    // every interpolated K is below max(K) (1 + 2^-23); the prefilter bound is
    // inflated by 2^-20 so that it covers them all
    P.Kmax_hi = (float)((double)kmax * (1.0 + std::ldexp(1.0, -20)));
    e = cudaMemcpy((void*)P.Ktab, K.data(), sizeof(float) * NGRID, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    // (16): the same table form with the e-O2+ reduced mass
    std::vector<float> Kr(NGRID, 0.0f);
    float krmax = 0.0f;
    if (have_recomb) {
        const double mur = g.m_e * g.m_OP / (g.m_e + g.m_OP);
        for (int i = 0; i < NGRID; ++i) {
            const double Ei = grid_energy(i);
            const double gv = std::sqrt(2.0 * QE * Ei / mur);
            Kr[i] = (float)(sigma_at(recomb, Ei) * gv);
            krmax = std::max(krmax, Kr[i]);
        }
    }
    P.have_recomb = have_recomb ? 1 : 0;
    P.Kmax_r_hi = (float)((double)krmax * (1.0 + std::ldexp(1.0, -20)));
    e = cudaMemcpy((void*)P.Ktab_r, Kr.data(), sizeof(float) * NGRID, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    // (22): the same table form with the e-O- reduced mass; its threshold
    std::vector<float> Kd(NGRID, 0.0f);
    float kdmax = 0.0f;
    if (have_edet) {
        const double mud = g.m_e * g.m_OM / (g.m_e + g.m_OM);
        for (int i = 0; i < NGRID; ++i) {
            const double Ei = grid_energy(i);
            const double gv = std::sqrt(2.0 * QE * Ei / mud);
            Kd[i] = (float)(sigma_at(edet, Ei) * gv);
            kdmax = std::max(kdmax, Kd[i]);
        }
    }
    P.have_edet = have_edet ? 1 : 0;
    P.thr_d = have_edet ? (float)edet.thr : 0.0f;
    P.Kmax_d_hi = (float)((double)kdmax * (1.0 + std::ldexp(1.0, -20)));
    e = cudaMemcpy((void*)P.Ktab_d, Kd.data(), sizeof(float) * NGRID, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    for (int s = 0; s < NSP; ++s) {
        int bps = 0;
        P.cum_smem[s] = 0;
        if (push_occupancy(s, P, &bps) || bps < 1) bps = 1;
        if (bps > MAX_PUSH_BLOCKS_PER_SM) bps = MAX_PUSH_BLOCKS_PER_SM;
        // the kinematics' table in shared memory when the blocks per SM stay
        if (cum_smem_allowed() && P.nproc[s] > 0 && (s == SP_E || ions_fused())) {
            int b2 = 0;
            P.cum_smem[s] = 1;
            if (push_occupancy(s, P, &b2) || std::min(b2, MAX_PUSH_BLOCKS_PER_SM) < bps) P.cum_smem[s] = 0;
        }
        c->grid_push[s] = std::max(bps * c->num_sms, min_push_blocks(P.sp[s].cap));
        P.push_warps[s] = (unsigned)c->grid_push[s] * (BLOCK / 32);
    }
    c->have_tables = true;
    c->dirty = true;
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_load_particles(o2pic_ctx* c, int species, const float* x, const float* vx, const float* vy,
                         const float* vz, const uint32_t* id, uint64_t n, int mem_kind, void* stream) {
    if (!c || species < 0 || species >= NSP) return O2PIC_E_INVALID_ARG;
    if (n > c->P.sp[species].cap) return O2PIC_E_INVALID_ARG;
    if (n > 0 && (!x || !vx || !vy || !vz || !id)) return O2PIC_E_INVALID_ARG;
    if (mem_kind != O2PIC_HOST && mem_kind != O2PIC_DEVICE) return O2PIC_E_INVALID_ARG;
    const unsigned next = 0;   // the check kernel raises it to max(id) + 1
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    c->latched = 0;
    cudaStream_t s = pick(c, stream);
    DevCtrl h;
    cudaError_t e = cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    const unsigned b = h.cur[species];
    const SpeciesBuf& B = c->P.sp[species];
    const cudaMemcpyKind k = (mem_kind == O2PIC_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (n > 0) {
        e = cudaMemcpyAsync(B.x[b], x, sizeof(float) * n, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.vx[b], vx, sizeof(float) * n, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.vy[b], vy, sizeof(float) * n, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.vz[b], vz, sizeof(float) * n, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.id[b], id, sizeof(uint32_t) * n, k, s);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    h.slots[species] = n;
    h.live[species] = n;
    h.removed[species] = 0;
    h.next_id[species] = next;
    h.error_flags = 0;
    e = cudaMemcpyAsync(c->d_ctrl, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (n > 0) {
        // both memory kinds: the particles are checked (and max(id) found) on
        // the device once they are there
        launch_load_check(species, c->P, n, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e);
        unsigned long long flags = 0;
        e = cudaMemcpy(&flags, &c->d_ctrl->error_flags, sizeof(flags), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e);
        if (flags & ERR_NONFINITE) {
            // leave the species empty (h.error_flags is 0)
            h.slots[species] = 0; h.live[species] = 0;
            e = cudaMemcpy(c->d_ctrl, &h, sizeof(h), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(c, e);
            return O2PIC_E_INVALID_ARG;
        }
    } else {
        e = cudaStreamSynchronize(s);   // the host arrays may be freed once we return
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    c->host_step = h.step;
    c->loaded[species] = true;
    c->flight_ok[species] = false;
    c->dirty = true;
    c->gen += 1;
    return O2PIC_OK;
}

static_assert(offsetof(DevCtrl, field_step) == offsetof(DevCtrl, step) + sizeof(unsigned long long),
              "o2pic_set_step writes step and field_step together");

int o2pic_set_step(o2pic_ctx* c, uint64_t step) {
    if (!c) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    const unsigned long long both[2] = {step, step};   // step and field_step (adjacent)
    cudaError_t e = cudaMemcpy(&c->d_ctrl->step, both, sizeof(both), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->host_step = step;
    c->dirty = true;
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_step(o2pic_ctx* c, uint64_t nsteps, void* stream) {
    if (!c) return O2PIC_E_INVALID_ARG;
    if (!c->have_tables) return O2PIC_E_STATE;
    if (c->latched) return c->latched;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e);
    cudaStream_t s = pick(c, stream);
    if (c->dirty) {
        int rc = prepare(c, s);
        if (rc) return rc;
    }
    for (uint64_t k = 0; k < nsteps; k += VRING / 2) {
        const unsigned long long n = std::min<unsigned long long>(nsteps - k, VRING / 2);
        if (int rc = fill_vring(c, c->host_step + 1, c->host_step + n, s)) return rc;
        enqueue_steps(c, n, s);
    }
    return cuda_fail(c, cudaGetLastError());
}

int o2pic_set_next_id(o2pic_ctx* c, int species, uint32_t next_id) {
    if (!c || species < 0 || species >= NSP) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    // the next id must not fall below the current one (after a load: the
    // largest loaded id + 1), or newborns would repeat live ids and share
    // their random streams
    unsigned long long cur = 0;
    cudaError_t e = cudaMemcpy(&cur, &c->d_ctrl->next_id[species], sizeof(cur), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if ((unsigned long long)next_id < cur) return O2PIC_E_INVALID_ARG;
    const unsigned long long v = next_id;
    e = cudaMemcpy(&c->d_ctrl->next_id[species], &v, sizeof(v), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_synchronize(o2pic_ctx* c) {
    if (!c) return O2PIC_E_INVALID_ARG;
    return sync_all(c);
}

int o2pic_read_particles(o2pic_ctx* c, int species, float* x, float* vx, float* vy, float* vz, uint32_t* id,
                         uint64_t cap, uint64_t* n, int mem_kind) {
    if (!c || species < 0 || species >= NSP || !n) return O2PIC_E_INVALID_ARG;
    if (mem_kind != O2PIC_HOST && mem_kind != O2PIC_DEVICE) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    cudaStream_t s = c->stream;
    DevCtrl h;
    cudaError_t e = cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    *n = h.live[species];
    const uint64_t m = std::min<uint64_t>(cap, h.live[species]);
    if (m == 0 || !x || !vx || !vy || !vz || !id) return rc;
    float *dx_ = x, *dvx = vx, *dvy = vy, *dvz = vz;
    uint32_t* did = id;
    std::vector<void*> tmp;
    if (mem_kind == O2PIC_HOST) {
        void* p;
        for (int k = 0; k < 5; ++k) {
            e = cudaMalloc(&p, 4 * m);
            if (e != cudaSuccess) { for (void* q : tmp) cudaFree(q); return cuda_fail(c, e); }
            tmp.push_back(p);
        }
        dx_ = (float*)tmp[0]; dvx = (float*)tmp[1]; dvy = (float*)tmp[2]; dvz = (float*)tmp[3]; did = (uint32_t*)tmp[4];
    }
    c->gepoch += 1;
    cudaMemsetAsync(c->d_gticket, 0, sizeof(unsigned), s);
    launch_gather(species, c->P, c->grid_compact, (1ull << 60) | c->gepoch, c->d_gticket, c->d_gflag, c->d_gval,
                  dx_, dvx, dvy, dvz, did, nullptr, m, c->d_gcount, s);
    c->launches += 1;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && mem_kind == O2PIC_HOST) {
        e = cudaMemcpy(x, dx_, 4 * m, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(vx, dvx, 4 * m, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(vy, dvy, 4 * m, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(vz, dvz, 4 * m, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(id, did, 4 * m, cudaMemcpyDeviceToHost);
    }
    for (void* q : tmp) cudaFree(q);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return check_flags(c);
}

int o2pic_set_majorant_cap(o2pic_ctx* c, const double* cap_eV) {
    if (!c || !cap_eV) return O2PIC_E_INVALID_ARG;
    for (int s = 0; s < NSP; ++s)
        if (!(cap_eV[s] > 0) && !std::isnan(cap_eV[s])) return O2PIC_E_INVALID_ARG;
    for (int s = 0; s < NSP; ++s) c->ecap[s] = std::isnan(cap_eV[s]) ? INFINITY : cap_eV[s];
    return O2PIC_OK;
}

int o2pic_set_coulomb(o2pic_ctx* c, uint32_t mask, double ln_lambda) {
    if (!c || mask > 63u || !(ln_lambda > 0.0) || !std::isfinite(ln_lambda)) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    Params& P = c->P;
    if (mask && !c->coul_alloc) {
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < NSP && e == cudaSuccess; ++s) {
            const unsigned long long cap = P.sp[s].cap;
            e = ctx_alloc(c, &P.csort[s], (size_t)cap);
            if (e == cudaSuccess) e = ctx_alloc(c, &P.chist[s], (size_t)(ceil_div(cap, TILE) + 1) * P.Nc);
            if (e == cudaSuccess) e = ctx_alloc(c, &P.ctot[s], (size_t)P.Nc);
            if (e == cudaSuccess) e = ctx_alloc(c, &P.cstart[s], (size_t)P.Nc);
        }
        if (e == cudaSuccess) e = configure_coulomb_smem(P.Nc);
        if (e != cudaSuccess) return cuda_fail(c, e);
        c->coul_alloc = true;
    }
    const o2pic_config& g = c->cfg;
    static const int pairs[6][2] = {{SP_E, SP_E}, {SP_OM, SP_OM}, {SP_OP, SP_OP}, {SP_E, SP_OP}, {SP_E, SP_OM},
                                    {SP_OM, SP_OP}};
    const double mass[NSP] = {g.m_e, g.m_OM, g.m_OP};
    const double dx = g.L / g.n_cells, dti = g.dt * (double)g.ion_subcycle;
    const double q4 = QE * QE * QE * QE;
    for (int r = 0; r < 6; ++r) {
        const double ma = mass[pairs[r][0]], mb = mass[pairs[r][1]];
        const double mu = ma * mb / (ma + mb);
        P.coul_K[r] = (float)(q4 * g.weight * ln_lambda * dti / (8.0 * M_PI * EPS0 * EPS0 * mu * mu * g.area * dx));
        P.coul_fa[r] = (float)(mb / (ma + mb));
        P.coul_fb[r] = (float)(ma / (ma + mb));
    }
    P.coul_mask = mask;
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_load_flight(o2pic_ctx* c, int species, const uint32_t* tc, uint64_t n, int mem_kind, void* stream) {
    if (!c || species < 0 || species >= NSP || (n > 0 && !tc)) return O2PIC_E_INVALID_ARG;
    if (mem_kind != O2PIC_HOST && mem_kind != O2PIC_DEVICE) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    DevCtrl h;
    cudaError_t e = cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    // only right after a load: every slot live, in load order
    if (h.slots[species] != n || h.live[species] != n) return O2PIC_E_INVALID_ARG;
    cudaStream_t s = pick(c, stream);
    if (n > 0) {
        e = cudaMemcpyAsync(c->P.sp[species].tc[h.cur[species]], tc, sizeof(uint32_t) * n,
                            mem_kind == O2PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    c->flight_ok[species] = true;
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_read_flight(o2pic_ctx* c, int species, uint32_t* tc, uint64_t cap, uint64_t* n, int mem_kind) {
    if (!c || species < 0 || species >= NSP || !n) return O2PIC_E_INVALID_ARG;
    if (mem_kind != O2PIC_HOST && mem_kind != O2PIC_DEVICE) return O2PIC_E_INVALID_ARG;
    if (c->dirty && c->have_tables) {
        // flights not drawn yet: draw them (as the next step would)
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e);
        int rc = prepare(c, c->stream);
        if (rc) return rc;
    }
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    cudaStream_t s = c->stream;
    DevCtrl h;
    cudaError_t e = cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    *n = h.live[species];
    const uint64_t m = std::min<uint64_t>(cap, h.live[species]);
    if (m == 0 || !tc) return rc;
    uint32_t* dtc = tc;
    void* tmp = nullptr;
    if (mem_kind == O2PIC_HOST) {
        e = cudaMalloc(&tmp, 4 * m);
        if (e != cudaSuccess) return cuda_fail(c, e);
        dtc = (uint32_t*)tmp;
    }
    c->gepoch += 1;
    cudaMemsetAsync(c->d_gticket, 0, sizeof(unsigned), s);
    launch_gather(species, c->P, c->grid_compact, (1ull << 60) | c->gepoch, c->d_gticket, c->d_gflag, c->d_gval,
                  nullptr, nullptr, nullptr, nullptr, nullptr, dtc, m, c->d_gcount, s);
    c->launches += 1;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && mem_kind == O2PIC_HOST) e = cudaMemcpy(tc, dtc, 4 * m, cudaMemcpyDeviceToHost);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return check_flags(c);
}

int o2pic_read_field(o2pic_ctx* c, double* phi, float* E) {
    if (!c) return O2PIC_E_INVALID_ARG;
    if (c->dirty && c->have_tables) {
        cudaSetDevice(c->device);
        int rc = prepare(c, c->stream);
        if (rc) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (phi) {
        e = cudaSetDevice(c->device);
        if (e == cudaSuccess) { launch_phi(c->P, c->last); e = cudaGetLastError(); }
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    if (phi) e = cudaMemcpy(phi, c->P.phi, sizeof(double) * c->P.Ng, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(E, c->P.Ef, sizeof(float) * c->P.Ng, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return rc;
}

int o2pic_read_currents(o2pic_ctx* c, uint64_t first, uint64_t n, double* out) {
    if (!c || (n && !out)) return O2PIC_E_INVALID_ARG;
    if (n == 0) return O2PIC_OK;
    const unsigned long long done = c->host_step;   // steps < done are complete
    if (c->dirty || first < c->ring_start || first + n > done || done - first > JRING - 1)
        return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    std::vector<unsigned long long> raw(JRING * NSP);
    cudaError_t e = cudaMemcpy(raw.data(), c->P.jring, sizeof(unsigned long long) * raw.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    const o2pic_config& g = c->cfg;
    const int charge[NSP] = {-1, -1, +1};
    const double unit = QE * g.weight / (256.0 * g.area * g.L);
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t k = first + i;
        double tot = 0.0;
        for (int s = 0; s < NSP; ++s) {
            const long long sum = (long long)raw[(k & (JRING - 1)) * NSP + s];
            const double J = (double)charge[s] * unit * (double)sum;
            out[5 * i + s] = J;
            tot += J;
        }
        const double v0 = g.U * std::sin(TWO_PI * g.f * ((double)k * g.dt));
        const double v1 = g.U * std::sin(TWO_PI * g.f * ((double)(k + 1) * g.dt));
        const double Jd = EPS0 * (v1 - v0) / (g.L * g.dt);
        out[5 * i + 3] = Jd;
        out[5 * i + 4] = tot + Jd;
    }
    return rc;
}

int o2pic_read_charge(o2pic_ctx* c, uint64_t* Q, uint64_t* Qacc, uint64_t* acc_steps) {
    if (!c) return O2PIC_E_INVALID_ARG;
    if (c->dirty && c->have_tables) {
        cudaSetDevice(c->device);
        int rc = prepare(c, c->stream);
        if (rc) return rc;
    }
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    const int Ng = c->P.Ng;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < NSP && e == cudaSuccess; ++s) {
        if (Q) e = cudaMemcpy(Q + (size_t)s * Ng, c->P.Q[s], 8 * (size_t)Ng, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && Qacc) e = cudaMemcpy(Qacc + (size_t)s * Ng, c->P.Qacc[s], 8 * (size_t)Ng, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && acc_steps) e = cudaMemcpy(acc_steps, &c->d_ctrl->acc_steps, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    return rc;
}

int o2pic_read_moments(o2pic_ctx* c, double* density, uint64_t* acc_steps, int reset) {
    if (!c) return O2PIC_E_INVALID_ARG;
    const int Ng = c->P.Ng;
    std::vector<uint64_t> Qa((size_t)NSP * Ng);
    uint64_t steps = 0;
    int rc = o2pic_read_charge(c, nullptr, Qa.data(), &steps);
    if (rc == O2PIC_E_CUDA) return rc;
    if (density) {
        const double dx = c->P.dx;
        for (int s = 0; s < NSP; ++s)
            for (int j = 0; j < Ng; ++j) {
                const double vol = c->cfg.area * ((j == 0 || j == Ng - 1) ? 0.5 * dx : dx);
                density[(size_t)s * Ng + j] =
                    steps ? (double)Qa[(size_t)s * Ng + j] / (65536.0 * (double)steps) * c->cfg.weight / vol : 0.0;
            }
    }
    if (acc_steps) *acc_steps = steps;
    if (reset) {
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < NSP && e == cudaSuccess; ++s) e = cudaMemset(c->P.Qacc[s], 0, 8 * (size_t)Ng);
        const unsigned long long zero = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&c->d_ctrl->acc_steps, &zero, 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return rc;
}

int o2pic_get_stats(o2pic_ctx* c, o2pic_stats* out) {
    if (!c || !out) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    DevCtrl h;
    cudaError_t e = cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    std::memset(out, 0, sizeof(*out));
    for (int s = 0; s < NSP; ++s) {
        for (int k = 0; k < MAXPROC; ++k) out->events[s][k] = h.cnt.events[s][k];
        out->absorbed[s][0] = h.cnt.absorbed[s][0];
        out->absorbed[s][1] = h.cnt.absorbed[s][1];
        out->born[s] = h.cnt.born[s];
        out->live[s] = h.live[s];
        out->slots[s] = h.slots[s];
        out->next_id[s] = h.next_id[s];
        out->particle_steps_species[s] = h.cnt.psteps[s];
    }
    out->neutralized = h.cnt.neutralized;
    out->pair_candidates = h.cnt.pair_candidates;
    out->particle_steps = h.cnt.particle_steps;
    out->warn_emax = h.cnt.warn_emax;
    out->warn_tries = h.cnt.warn_tries;
    out->warn_pair_gt1 = h.cnt.warn_pair_gt1;
    out->id_overflow = h.cnt.id_overflow;
    out->recombined = h.cnt.recombined;
    out->rec_candidates = h.cnt.rec_candidates;
    out->edetached = h.cnt.edetached;
    out->edet_candidates = h.cnt.edet_candidates;
    out->coulomb_pairs = h.cnt.coulomb_pairs;
    out->warn_numax = h.cnt.warn_numax;
    out->step = h.step;
    out->error_flags = h.error_flags;
    return rc;
}

int o2pic_set_timing(o2pic_ctx* c, int on) {
    if (!c) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    c->timing = on != 0;
    for (int k = 0; k < NKK; ++k) { c->ms[k] = 0; c->nlaunch[k] = 0; }
    return rc == O2PIC_E_CUDA ? rc : O2PIC_OK;
}

int o2pic_get_timing(o2pic_ctx* c, double* ms, uint64_t* launches, uint64_t* items, int nkinds) {
    if (!c || nkinds < 0) return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    for (int k = 0; k < nkinds && k < NKK; ++k) {
        if (ms) ms[k] = c->ms[k];
        if (launches) launches[k] = c->nlaunch[k];
        if (items) items[k] = 0;
    }
    return rc == O2PIC_E_CUDA ? rc : O2PIC_OK;
}

uint64_t o2pic_launch_count(o2pic_ctx* c) { return c ? c->launches : 0; }

int o2pic_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, uint64_t n, void* stream) {
    if ((!ctr || !key || !out) && n) return O2PIC_E_INVALID_ARG;
    if (n == 0) return O2PIC_OK;
    launch_philox(ctr, key, out, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

int o2pic_ln_f32(const float* x, float* out, uint64_t n, void* stream) {
    if ((!x || !out) && n) return O2PIC_E_INVALID_ARG;
    if (n == 0) return O2PIC_OK;
    launch_ln(x, out, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

// ============================================================ batched stepping
}  // extern "C"

struct o2pic_batch {
    std::vector<o2pic_ctx*> ctx;
    uint64_t K = 0;                       // steps per graph replay
    int device = 0;
    cudaStream_t stream = nullptr;        // origin stream: ring fills and graph launches
    std::vector<cudaStream_t> branch;     // one capture branch per context
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned long long> launches_per_replay;
    std::vector<unsigned long long> phase_step;   // host_step of each context at capture
    std::vector<unsigned long long> gen;          // generation of each context at capture
    // fused mode: one batched launch per kernel and step for all contexts
    bool fused = false, fusable = false;
    Params* dP = nullptr;                 // [n] parameters of each context
    PairSpec* dR = nullptr;               // [n] (16) of each context
    PairSpec* dD = nullptr;               // [n] (22)
    PairSpec* dN = nullptr;               // [n] (17)
    uint4* dmap = nullptr;                // block maps, concatenated
    size_t map_push[NSP] = {0, 0, 0}, map_comp[NSP] = {0, 0, 0}, map_rh = 0, map_rp = 0, map_nh = 0, map_np = 0;
    size_t map_dh = 0, map_dp = 0;
    int nb_push[NSP] = {0, 0, 0}, nb_comp[NSP] = {0, 0, 0}, nb_rh = 0, nb_rp = 0, nb_nh = 0, nb_np = 0;
    int nb_dh = 0, nb_dp = 0;
    bool any_recomb = false, any_neutral = false, any_edet = false;
    size_t smem_push = 0, smem_field = 0, smem_hist = 0;
};

namespace {

void batch_release_graph(o2pic_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Device tables of the fused mode: each context's Params and PairSpecs, and
// the block maps (discharge, block, blocks) of every batched launch.
int fused_tables(o2pic_batch* b) {
    const size_t n = b->ctx.size();
    std::vector<Params> hp(n);
    std::vector<PairSpec> hr(n), hn(n), hd(n);
    std::vector<uint4> map;
    auto add_map = [&](size_t& off, int& nb, auto blocks_of) {
        off = map.size();
        for (size_t i = 0; i < n; ++i) {
            const unsigned k = (unsigned)blocks_of(b->ctx[i]);
            for (unsigned j = 0; j < k; ++j) map.push_back(make_uint4((unsigned)i, j, k, 0u));
        }
        nb = (int)(map.size() - off);
    };
    auto tiles = [](unsigned long long cap) { return std::max<unsigned long long>(1, ceil_div(cap, TILE)); };
    b->any_recomb = b->any_neutral = b->any_edet = false;
    b->smem_push = b->smem_field = b->smem_hist = 0;
    for (size_t i = 0; i < n; ++i) {
        o2pic_ctx* c = b->ctx[i];
        const Params& P = c->P;
        hp[i] = P;
        hr[i] = spec_rec(c);
        hn[i] = spec_neu(c);
        hd[i] = spec_edet(c);
        b->any_recomb |= P.have_recomb != 0;
        b->any_edet |= P.have_edet != 0;
        b->any_neutral |= P.have_neutral != 0;
        for (int sp = 0; sp < NSP; ++sp) b->smem_push = std::max(b->smem_push, push_smem_bytes(sp, P));
        b->smem_field = std::max(b->smem_field, field_smem_bytes(P));
        b->smem_hist = std::max(b->smem_hist, 3 * sizeof(unsigned) * (size_t)P.Nc);
    }
    for (int sp = 0; sp < NSP; ++sp) {
        add_map(b->map_push[sp], b->nb_push[sp], [&](o2pic_ctx* c) { return c->grid_push[sp]; });
        add_map(b->map_comp[sp], b->nb_comp[sp],
                [&](o2pic_ctx* c) { return std::min<unsigned long long>(tiles(c->P.sp[sp].cap), 16); });
    }
    add_map(b->map_dh, b->nb_dh, [&](o2pic_ctx* c) {
        return std::min<unsigned long long>(tiles(c->P.sp[SP_OM].cap) + tiles(c->P.sp[SP_E].cap), 32); });
    add_map(b->map_dp, b->nb_dp, [&](o2pic_ctx* c) { return std::min<unsigned long long>(tiles(c->P.sp[SP_OM].cap), 64); });
    add_map(b->map_rh, b->nb_rh, [&](o2pic_ctx* c) {
        return std::min<unsigned long long>(tiles(c->P.sp[SP_E].cap) + tiles(c->P.sp[SP_OP].cap), 32); });
    add_map(b->map_rp, b->nb_rp, [&](o2pic_ctx* c) { return std::min<unsigned long long>(tiles(c->P.sp[SP_E].cap), 64); });
    add_map(b->map_nh, b->nb_nh, [&](o2pic_ctx* c) {
        return std::min<unsigned long long>(tiles(c->P.sp[SP_OM].cap) + tiles(c->P.sp[SP_OP].cap), 32); });
    add_map(b->map_np, b->nb_np, [&](o2pic_ctx* c) { return std::min<unsigned long long>(tiles(c->P.sp[SP_OM].cap), 64); });
    if (b->dP) cudaFree(b->dP);
    if (b->dR) cudaFree(b->dR);
    if (b->dD) cudaFree(b->dD);
    if (b->dN) cudaFree(b->dN);
    if (b->dmap) cudaFree(b->dmap);
    b->dP = nullptr; b->dR = b->dN = b->dD = nullptr; b->dmap = nullptr;
    if (cudaMalloc((void**)&b->dP, sizeof(Params) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->dR, sizeof(PairSpec) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->dD, sizeof(PairSpec) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->dN, sizeof(PairSpec) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->dmap, sizeof(uint4) * std::max<size_t>(map.size(), 1)) != cudaSuccess)
        return O2PIC_E_CUDA;
    if (cudaMemcpy(b->dP, hp.data(), sizeof(Params) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dR, hr.data(), sizeof(PairSpec) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dD, hd.data(), sizeof(PairSpec) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dN, hn.data(), sizeof(PairSpec) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dmap, map.data(), sizeof(uint4) * map.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return O2PIC_E_CUDA;
    return O2PIC_OK;
}

// The fused kernel sequence of K steps on stream s (contexts share the
// schedule: ion subcycle, compaction period and their phases).
void enqueue_fused(o2pic_batch* b, cudaStream_t s) {
    o2pic_ctx* c0 = b->ctx[0];
    const unsigned S = (unsigned)c0->cfg.ion_subcycle;
    const int n = (int)b->ctx.size();
    unsigned long long step = c0->host_step;
    unsigned since = c0->since_check;
    unsigned long long launches = 0;
    for (uint64_t k = 0; k < b->K; ++k) {
        const bool ion = (step % S) == 0;
        launch_push_batched(SP_E, b->dP, b->dmap + b->map_push[SP_E], b->nb_push[SP_E], b->smem_push, s);
        launches += 1;
        if (ion) {
            for (int sp = SP_OM; sp <= SP_OP; ++sp) {
                launch_push_batched(sp, b->dP, b->dmap + b->map_push[sp], b->nb_push[sp], b->smem_push, s);
                launches += 1;
                if (!ions_fused()) {
                    launch_filter_batched(sp, b->dP, b->dmap + b->map_push[sp], b->nb_push[sp], s);
                    launch_cand_batched(sp, b->dP, b->dmap + b->map_push[sp], b->nb_push[sp], s);
                    launches += 2;
                }
            }
            if (b->any_edet) {
                launch_pair_hist_batched(b->dP, b->dD, b->dmap + b->map_dh, b->nb_dh, b->smem_hist, s);
                launch_pair_batched(b->dP, b->dD, b->dmap + b->map_dp, b->nb_dp, s);
                launch_edet_apply_batched(b->dP, b->dD, n, s);
                launches += 3;
            }
            if (b->any_recomb) {
                launch_pair_hist_batched(b->dP, b->dR, b->dmap + b->map_rh, b->nb_rh, b->smem_hist, s);
                launch_pair_batched(b->dP, b->dR, b->dmap + b->map_rp, b->nb_rp, s);
                launch_pair_apply_batched(b->dP, b->dR, n, s);
                launches += 3;
            }
            if (b->any_neutral) {
                launch_pair_hist_batched(b->dP, b->dN, b->dmap + b->map_nh, b->nb_nh, b->smem_hist, s);
                launch_pair_batched(b->dP, b->dN, b->dmap + b->map_np, b->nb_np, s);
                launches += 2;
            }
        }
        launch_field_batched(b->dP, n, b->smem_field, 0, ion ? 7 : 1, s);
        launches += 1;
        step += 1;
        if (++since >= c0->cfg.compact_check) {
            for (int sp = 0; sp < NSP; ++sp)
                launch_compact_batched(sp, b->dP, b->dmap + b->map_comp[sp], b->nb_comp[sp], s);
            launches += 3;
            since = 0;
        }
    }
    for (o2pic_ctx* c : b->ctx) { c->host_step = step; c->since_check = since; c->launches += launches; }
}

// Records K steps of every context into a graph: in fused mode one batched
// launch per kernel and step, else one branch per context.  Nothing runs;
// the contexts' host counters are restored afterwards.
int batch_capture(o2pic_batch* b) {
    batch_release_graph(b);
    if (b->fused)
        if (int rc = fused_tables(b)) return rc;
    const size_t n = b->ctx.size();
    std::vector<unsigned long long> hs(n), launches(n), nl(n * NKK);
    std::vector<unsigned> sc(n);
    for (size_t i = 0; i < n; ++i) {
        o2pic_ctx* c = b->ctx[i];
        hs[i] = c->host_step; sc[i] = c->since_check; launches[i] = c->launches;
        for (int k = 0; k < NKK; ++k) nl[i * NKK + k] = c->nlaunch[k];
    }
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return O2PIC_E_CUDA;
    if (b->fused) {
        enqueue_fused(b, b->stream);
    } else {
        // several branches: no early-launched blocks that could crowd out
        // the single-block kernels of other branches
        pdl_enabled = O2PIC_GRAPH_PDL_SINGLE && n == 1;
        cudaEventRecord(b->fork, b->stream);
        for (size_t i = 0; i < n; ++i) {
            cudaStreamWaitEvent(b->branch[i], b->fork, 0);
            enqueue_steps(b->ctx[i], b->K, b->branch[i]);
            cudaEventRecord(b->join[i], b->branch[i]);
            cudaStreamWaitEvent(b->stream, b->join[i], 0);
        }
        pdl_enabled = true;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    for (size_t i = 0; i < n; ++i) {
        o2pic_ctx* c = b->ctx[i];
        b->launches_per_replay[i] = c->launches - launches[i];
        b->phase_step[i] = hs[i];
        b->gen[i] = c->gen;
        c->host_step = hs[i]; c->since_check = sc[i]; c->launches = launches[i];
        for (int k = 0; k < NKK; ++k) c->nlaunch[k] = nl[i * NKK + k];
    }
    if (ec != cudaSuccess || e != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); cudaGetLastError(); return O2PIC_E_CUDA; }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) { batch_release_graph(b); cudaGetLastError(); return O2PIC_E_CUDA; }
    return O2PIC_OK;
}

// Live-slot count of each species of a context (device control block).
int ctx_slots(o2pic_ctx* c, unsigned long long slots[NSP]) {
    DevCtrl h;
    if (cudaMemcpy(&h, c->d_ctrl, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(c, cudaErrorUnknown);
    for (int s = 0; s < NSP; ++s) slots[s] = h.slots[s];
    return O2PIC_OK;
}

int default_push_blocks(o2pic_ctx* c, int s) {
    int bps = 0;
    if (push_occupancy(s, c->P, &bps) || bps < 1) bps = 1;
    if (bps > MAX_PUSH_BLOCKS_PER_SM) bps = MAX_PUSH_BLOCKS_PER_SM;
    return std::max(bps * c->num_sms, min_push_blocks(c->P.sp[s].cap));
}

}  // namespace

extern "C" {

int o2pic_set_launch_shape(o2pic_ctx* c, const int32_t push_blocks[3]) {
    if (!c || !push_blocks) return O2PIC_E_INVALID_ARG;
    if (!c->have_tables) return O2PIC_E_STATE;
    for (int s = 0; s < NSP; ++s)
        if (push_blocks[s] < min_push_blocks(c->P.sp[s].cap) || push_blocks[s] > MAX_PUSH_BLOCKS_PER_SM * c->num_sms)
            return O2PIC_E_INVALID_ARG;
    int rc = sync_all(c);
    if (rc == O2PIC_E_CUDA) return rc;
    for (int s = 0; s < NSP; ++s) {
        c->grid_push[s] = push_blocks[s];
        c->P.push_warps[s] = (unsigned)push_blocks[s] * (BLOCK / 32);
    }
    c->gen += 1;
    return O2PIC_OK;
}

int o2pic_get_launch_shape(o2pic_ctx* c, int32_t push_blocks[3]) {
    if (!c || !push_blocks) return O2PIC_E_INVALID_ARG;
    for (int s = 0; s < NSP; ++s) push_blocks[s] = c->grid_push[s];
    return O2PIC_OK;
}

int o2pic_batch_create(o2pic_ctx* const* ctxs, int32_t n, uint64_t K, o2pic_batch** out) {
    if (!out) return O2PIC_E_INVALID_ARG;
    *out = nullptr;
    if (!ctxs || n < 1 || K < 1 || K > VRING / 2) return O2PIC_E_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        o2pic_ctx* c = ctxs[i];
        if (!c || c->device != ctxs[0]->device) return O2PIC_E_INVALID_ARG;
        if (K % (uint64_t)c->cfg.ion_subcycle || K % (uint64_t)c->cfg.compact_check) return O2PIC_E_INVALID_ARG;
        if (!c->have_tables) return O2PIC_E_STATE;
        if (c->latched) return c->latched;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return O2PIC_E_INVALID_ARG;
    }
    if (cudaSetDevice(ctxs[0]->device) != cudaSuccess) return O2PIC_E_CUDA;
    o2pic_batch* b = new (std::nothrow) o2pic_batch;
    if (!b) return O2PIC_E_CUDA;
    b->ctx.assign(ctxs, ctxs + n);
    b->K = K;
    b->device = ctxs[0]->device;
    b->branch.assign(n, nullptr);
    b->join.assign(n, nullptr);
    b->launches_per_replay.assign(n, 0);
    b->phase_step.assign(n, 0);
    b->gen.assign(n, 0);
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&b->t0) == cudaSuccess && cudaEventCreate(&b->t1) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i)
        ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { o2pic_batch_destroy(b); return O2PIC_E_CUDA; }
    // initial deposit and field of contexts not yet stepped; timing off (no
    // event records inside the graph)
    for (o2pic_ctx* c : b->ctx) {
        int rc = sync_all(c);
        if (rc) { o2pic_batch_destroy(b); return rc; }
        if (c->timing) o2pic_set_timing(c, 0);
        if (c->dirty) {
            rc = prepare(c, b->stream);
            if (!rc) rc = cuda_fail(c, cudaStreamSynchronize(b->stream));
            if (rc) { o2pic_batch_destroy(b); return rc; }
        }
    }
    // fused when several contexts share the step schedule and its phase (one
    // context runs its own kernels directly)
    b->fused = n > 1;
    for (o2pic_ctx* c : b->ctx) {
        const o2pic_ctx* c0 = b->ctx[0];
        if (c->cfg.ion_subcycle != c0->cfg.ion_subcycle || c->cfg.compact_check != c0->cfg.compact_check ||
            c->host_step % (unsigned long long)c->cfg.ion_subcycle !=
                c0->host_step % (unsigned long long)c0->cfg.ion_subcycle ||
            c->since_check != c0->since_check)
            b->fused = false;
    }
    if (const char* env = std::getenv("O2PIC_BATCH_BRANCHES")) if (env[0] == '1') b->fused = false;
    // the Coulomb collisions have no batched launches: their contexts get branches
    for (o2pic_ctx* c : b->ctx) if (c->P.coul_mask) b->fused = false;
    b->fusable = b->fused;
    int rc = batch_capture(b);
    if (rc) { o2pic_batch_destroy(b); return rc; }
    *out = b;
    return O2PIC_OK;
}

int o2pic_batch_step(o2pic_batch* b, uint64_t launches) {
    if (!b || !b->exec) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return O2PIC_E_CUDA;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        o2pic_ctx* c = b->ctx[i];
        if (c->latched) return c->latched;
        // the graph holds the kernel sequence of its capture phase, with the
        // context's tables, launch shape and particle buffers of that time
        if ((c->host_step - b->phase_step[i]) % b->K || c->gen != b->gen[i] || c->dirty) return O2PIC_E_STATE;
    }
    for (uint64_t r = 0; r < launches; ++r) {
        for (o2pic_ctx* c : b->ctx)
            if (int rc = fill_vring(c, c->host_step + 1, c->host_step + b->K, b->stream)) return rc;
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return O2PIC_E_CUDA;
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            o2pic_ctx* c = b->ctx[i];
            c->host_step += b->K;
            c->launches += b->launches_per_replay[i];
            c->last = b->stream;
        }
    }
    return O2PIC_OK;
}

void* o2pic_batch_stream(o2pic_batch* b) { return b ? (void*)b->stream : nullptr; }

int o2pic_batch_synchronize(o2pic_batch* b) {
    if (!b) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return O2PIC_E_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return O2PIC_E_CUDA;
    int first = O2PIC_OK;
    for (o2pic_ctx* c : b->ctx) {
        const int rc = check_flags(c);
        if (rc && !first) first = rc;
    }
    return first;
}

int o2pic_batch_autotune(o2pic_batch* b, o2pic_tune_report* report) {
    if (!b) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return O2PIC_E_CUDA;
    if (int rc = o2pic_batch_synchronize(b)) return rc;
    static const int32_t policies[] = {0, 256, 512, 1024, 2048, 4096, 8192};
    const int np = (int)(sizeof(policies) / sizeof(policies[0]));
    o2pic_tune_report rep;
    std::memset(&rep, 0, sizeof(rep));
    const size_t n = b->ctx.size();
    std::vector<std::vector<int32_t>> shapes(np, std::vector<int32_t>(3 * n));
    for (size_t i = 0; i < n; ++i) {
        o2pic_ctx* c = b->ctx[i];
        unsigned long long slots[NSP];
        if (int rc = ctx_slots(c, slots)) return rc;
        for (int p = 0; p < np; ++p)
            for (int s = 0; s < NSP; ++s) {
                long long g;
                if (policies[p] == 0) g = default_push_blocks(c, s);
                else g = (long long)((slots[s] + (unsigned long long)policies[p] * (BLOCK / 32) - 1) /
                                     ((unsigned long long)policies[p] * (BLOCK / 32)));
                g = std::max<long long>(min_push_blocks(c->P.sp[s].cap),
                                        std::min<long long>(g, (long long)MAX_PUSH_BLOCKS_PER_SM * c->num_sms));
                shapes[p][3 * i + s] = (int32_t)g;
            }
    }
    int best = 0;
    double best_ms = 0.0;
    for (int p = 0; p < np; ++p) {
        for (size_t i = 0; i < n; ++i)
            if (int rc = o2pic_set_launch_shape(b->ctx[i], &shapes[p][3 * i])) return rc;
        if (int rc = batch_capture(b)) return rc;
        if (cudaGraphUpload(b->exec, b->stream) != cudaSuccess) return O2PIC_E_CUDA;
        for (o2pic_ctx* c : b->ctx)
            if (int rc = fill_vring(c, c->host_step + 1, c->host_step + b->K, b->stream)) return rc;
        cudaEventRecord(b->t0, b->stream);
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return O2PIC_E_CUDA;
        cudaEventRecord(b->t1, b->stream);
        for (size_t i = 0; i < n; ++i) {
            b->ctx[i]->host_step += b->K;
            b->ctx[i]->launches += b->launches_per_replay[i];
        }
        if (int rc = o2pic_batch_synchronize(b)) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->t0, b->t1);
        if (rep.n < O2PIC_TUNE_MAX) {
            rep.particles_per_warp[rep.n] = policies[p];
            rep.ms[rep.n] = ms;
            rep.n += 1;
        }
        if (p == 0 || ms < best_ms) { best = p; best_ms = ms; }
    }
    for (size_t i = 0; i < n; ++i)
        if (int rc = o2pic_set_launch_shape(b->ctx[i], &shapes[best][3 * i])) return rc;
    // with a shared schedule, also the other launch mode at the best shape
    if (b->fusable) {
        b->fused = !b->fused;
        if (int rc = batch_capture(b)) return rc;
        if (cudaGraphUpload(b->exec, b->stream) != cudaSuccess) return O2PIC_E_CUDA;
        for (o2pic_ctx* c : b->ctx)
            if (int rc = fill_vring(c, c->host_step + 1, c->host_step + b->K, b->stream)) return rc;
        cudaEventRecord(b->t0, b->stream);
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return O2PIC_E_CUDA;
        cudaEventRecord(b->t1, b->stream);
        for (size_t i = 0; i < n; ++i) {
            b->ctx[i]->host_step += b->K;
            b->ctx[i]->launches += b->launches_per_replay[i];
        }
        if (int rc = o2pic_batch_synchronize(b)) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->t0, b->t1);
        rep.other_mode_ms = ms;
        if (!(ms < best_ms)) b->fused = !b->fused;   // keep the faster mode
    }
    if (int rc = batch_capture(b)) return rc;
    rep.chosen = best;
    rep.fused = b->fused ? 1 : 0;
    if (report) *report = rep;
    return O2PIC_OK;
}

void o2pic_batch_destroy(o2pic_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_release_graph(b);
    for (cudaStream_t s : b->branch) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->stream) cudaStreamDestroy(b->stream);
    for (void* p : {(void*)b->dP, (void*)b->dR, (void*)b->dN, (void*)b->dD, (void*)b->dmap}) if (p) cudaFree(p);
    delete b;
}

}  // extern "C"

