// o2pic oracle — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, sequential CPU implementation of one time step of the
// 1D3V particle-in-cell Monte-Carlo-collision (PIC-MCC) model of a
// capacitively coupled RF oxygen discharge (Bronold et al., "Particle-based
// modeling of oxygen discharges", ICPIG 2007, Sec. 2).  It exists to check the
// CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
// / reference legs may load it.  It shares no code with the CUDA library: the
// two are written separately from the same readings of the paper.
//
// Everything is ordinary loops over std::vectors in the order the method
// states.  The per-particle loop of a species and the deposit may run on
// several host threads (OpenMP, oracle_set_threads; 1 by default): each
// particle's update depends on nothing but itself and the field, every
// thread keeps its own counters and births over a contiguous range of
// particles, and the ranges are merged in particle order, so the results are
// those of one thread bit for bit.  The particle arithmetic is templated on the precision R:
//   R = float  : "mirror" mode, the precision the method fixes for particles
//                (FP32 particles, FP64 Poisson); used for per-particle parity.
//   R = double : FP64 reference, used to state the error of the FP32 results.
// The Poisson solve and the charge reduction are always FP64 / exact integer.
//
// Paper passages followed (Sec. 2 unless stated):
//   * one spatial coordinate 0 <= x <= L, all three velocity components kept;
//   * one electrode driven by U sin(2 pi f t), the other grounded;
//   * both electrodes totally absorbing, no secondary emission;
//   * O2 background at n = p / kT, T = 300 K; metastable O2(a) at n_D = C n_O2;
//   * collisions decoupled from free flights, collision time and type from
//     kinetic considerations (null-collision Monte Carlo);
//   * three kinetic species e, O-, O2+; reactions of Table 1;
//   * Eq. 1 (associative detachment) and the Landau-Zener sigma_n enter as
//     cross-section data;
//   * ion-ion neutralization (17) as a binary, cell-local (DSMC-like) process.
// Where the paper is silent a reading is taken and stated beside the code
// that implements it (leapfrog, CIC, the Poisson discretization, isotropic
// scattering, birth velocities, pairing).
//
// Parity status of each function is stated next to it.  All functions here
// are pinned by tests under tests/ (closed forms, invariants, brute force);
// the coupled discharge against the paper's figures is NOT pinned (the paper's
// cross sections are unpublished).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>
#include <limits>
#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- constants
// CODATA 2018 exact / recommended values (SI).
const double QE = 1.602176634e-19;     // elementary charge [C]
const double KB = 1.380649e-23;        // Boltzmann constant [J/K]
const double EPS0 = 8.8541878128e-12;  // vacuum permittivity [F/m]
const double TWO_PI = 6.283185307179586476925286766559;

enum { SP_E = 0, SP_OM = 1, SP_OP = 2, NSP = 3 };
enum { K_ELASTIC = 0, K_EXCITE = 1, K_IONIZE = 2, K_ATTACH = 3, K_DETACH = 4, K_CX = 5, K_NEUTRALIZE = 6,
       K_RECOMBINE = 7, K_EDETACH = 8 };
enum { T_O2 = 0, T_O2_META = 1, T_ION = 2, T_ELECTRON = 3 };

// Energy grid of the rate tables: 32 points per octave on [2^-10, 2^12] eV.
const int GRID_OCT_LO = -10;
const int GRID_OCTAVES = 22;
const int GRID_SUB = 32;
const int NGRID = GRID_OCTAVES * GRID_SUB + 1;   // 705 points, last = 2^12 eV
const int MAXPROC = 16;
const int MAX_TRIES = 32;                        // rejection-loop cap
const double FIX_ONE = 65536.0;                  // CIC fixed point: 2^16 per particle

// RNG stream tags (counter word 1).  TAG_FLIGHT + s: the first free-flight
// draw of a particle of species s (at load or birth).
enum { TAG_E = 0, TAG_OM = 1, TAG_OP = 2, TAG_PAIR = 3, TAG_SHIFT = 4, TAG_REC = 5, TAG_SHIFT_REC = 6,
       TAG_FLIGHT = 7, TAG_EDET = 10, TAG_SHIFT_EDET = 11, TAG_COUL = 12, TAG_SHIFT_COUL = 18 };

// Coulomb reactions (1)-(6) of Table 1: (species a, species b).
const int COUL_PAIRS[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 2}, {0, 1}, {1, 2}};

// ------------------------------------------------------------------ Philox
// Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11: 10 rounds of the Philox S-box with multipliers
// 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
struct U4 { uint32_t v[4]; };

U4 philox4x32_10(const uint32_t ctr[4], const uint32_t key[2]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    U4 r; r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

// Sequential words of the stream keyed by (key0, seed) with counter
// (step_lo, tag, block, step_hi); block b yields words 4b..4b+3.
struct Stream {
    uint32_t key[2];
    uint32_t ctr[4];
    U4 buf;
    int pos;      // next word inside buf (4 = exhausted)
    Stream(uint32_t key0, uint32_t seed, uint64_t step, uint32_t tag) {
        key[0] = key0; key[1] = seed;
        ctr[0] = (uint32_t)step; ctr[1] = tag; ctr[2] = 0; ctr[3] = (uint32_t)(step >> 32);
        buf = philox4x32_10(ctr, key);
        pos = 0;
    }
    uint32_t next() {
        if (pos == 4) { ctr[2] += 1; buf = philox4x32_10(ctr, key); pos = 0; }
        return buf.v[pos++];
    }
};

// u32 -> uniform on [0, 1) with 24 random bits (exact in float and double).
template <class R> R uniform(uint32_t w) { return (R)(w >> 8) * (R)(1.0 / 16777216.0); }

// --------------------------------------------------------------- math (R)
inline float fma_(float a, float b, float c) { return std::fmaf(a, b, c); }
inline double fma_(double a, double b, double c) { return std::fma(a, b, c); }
inline float sqrt_(float a) { return std::sqrt(a); }
inline double sqrt_(double a) { return std::sqrt(a); }

// Natural log in single precision by the atanh series (Abramowitz & Stegun
// 4.1.27): x = 2^e m, m in [sqrt(1/2), sqrt(2)), t = (m-1)/(m+1),
// ln m = 2 t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9).  |t| <= 0.1716, so the
// truncated tail is below 3e-9 relative.  Used only for x in (0, 1] (the
// polar normal method).  Written here from the series; the CUDA path has
// its own implementation of the same series so that both produce identical
// single-precision normals.
float ln_(float x) {
    int e;
    float m = std::frexp(x, &e);   // x = m 2^e, m in [0.5, 1)
    m = m * 2.0f; e -= 1;          // m in [1, 2)
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    float t = (m - 1.0f) / (m + 1.0f);
    float t2 = t * t;
    float p = fma_(t2, 0.111111111f, 0.142857143f);
    p = fma_(t2, p, 0.2f);
    p = fma_(t2, p, 0.333333333f);
    p = fma_(t2, p, 1.0f);
    float lnm = (2.0f * t) * p;
    return fma_((float)e, 0.693147182f, lnm);
}
double ln_(double x) { return std::log(x); }

template <class R> R dot3(R ax, R ay, R az, R bx, R by, R bz) {
    return fma_(ax, bx, fma_(ay, by, az * bz));
}

// Marsaglia (1972) point on the unit sphere from a uniform point of the unit
// disk: (a, b), s = a^2 + b^2 < 1  ->  (2a sqrt(1-s), 2b sqrt(1-s), 1 - 2s).
template <class R> void isotropic(Stream& st, R n[3], uint64_t& warn) {
    for (int t = 0; t < MAX_TRIES; ++t) {
        R a = (R)2 * uniform<R>(st.next()) - (R)1;
        R b = (R)2 * uniform<R>(st.next()) - (R)1;
        R s = fma_(a, a, b * b);
        if (s < (R)1) {
            R h = (R)2 * sqrt_((R)1 - s);
            n[0] = a * h; n[1] = b * h; n[2] = (R)1 - (R)2 * s;
            return;
        }
    }
    warn += 1; n[0] = 0; n[1] = 0; n[2] = 1;
}

// Marsaglia-Bray polar method: a pair of independent standard normals.
template <class R> void normal_pair(Stream& st, R& z0, R& z1, uint64_t& warn) {
    for (int t = 0; t < MAX_TRIES; ++t) {
        R a = (R)2 * uniform<R>(st.next()) - (R)1;
        R b = (R)2 * uniform<R>(st.next()) - (R)1;
        R s = fma_(a, a, b * b);
        if (s > (R)0 && s < (R)1) {
            R f = sqrt_(((R)(-2) * ln_(s)) / s);
            z0 = a * f; z1 = b * f;
            return;
        }
    }
    warn += 1; z0 = 0; z1 = 0;
}

// Three Maxwellian velocity components with standard deviation sig.
template <class R> void maxwellian(Stream& st, R sig, R v[3], uint64_t& warn) {
    R z0, z1, z2, z3;
    normal_pair<R>(st, z0, z1, warn);
    normal_pair<R>(st, z2, z3, warn);
    v[0] = sig * z0; v[1] = sig * z1; v[2] = sig * z2;
}

// ------------------------------------------------------------ rate tables
// Grid point i: E_i = 2^(i/32 - 10) (1 + (i mod 32)/32) eV.
double grid_energy(int i) {
    int oct = i / GRID_SUB, sub = i % GRID_SUB;
    return std::ldexp(1.0 + sub / (double)GRID_SUB, oct + GRID_OCT_LO);
}

// Position of E on the grid: index i and weight w in [0,1) with
// E = E_i + w (E_{i+1} - E_i).  Exact in float and double (frexp/ldexp are
// exact, 32 f and its floor are exact).  E below the grid -> point 0;
// E at or above 2^12 eV -> last point (flagged by the caller).
template <class R> void grid_locate(R E, int& i, R& w, bool& above) {
    above = false;
    if (!(E >= (R)std::ldexp(1.0, GRID_OCT_LO))) { i = 0; w = 0; return; }
    if (E >= (R)std::ldexp(1.0, GRID_OCT_LO + GRID_OCTAVES)) { i = NGRID - 1; w = 0; above = true; return; }
    int ex;
    R m = std::frexp(E, &ex);           // E = m 2^ex, m in [0.5,1)
    R f = m * (R)2 - (R)1;              // E = 2^(ex-1) (1+f)
    R f32 = f * (R)GRID_SUB;
    R fl = std::floor(f32);
    i = (ex - 1 - GRID_OCT_LO) * GRID_SUB + (int)fl;
    w = f32 - fl;
}

// Piecewise-linear value of table T (stride `stride`, column k) at E.
template <class R> R grid_interp(const std::vector<R>& T, int stride, int k, int i, R w) {
    if (i >= NGRID - 1) return T[(size_t)(NGRID - 1) * stride + k];
    R a = T[(size_t)i * stride + k], b = T[(size_t)(i + 1) * stride + k];
    return fma_(w, b - a, a);
}

// Linear interpolation of a user (E, sigma) table, constant beyond its ends,
// zero below the process threshold.
double sigma_at(const std::vector<double>& Et, const std::vector<double>& st, double thr, double E) {
    if (E < thr) return 0.0;
    size_t n = Et.size();
    if (E <= Et[0]) return st[0];
    if (E >= Et[n - 1]) return st[n - 1];
    size_t b = std::upper_bound(Et.begin(), Et.end(), E) - Et.begin();
    double Ea = Et[b - 1], Eb = Et[b], sa = st[b - 1], sb = st[b];
    return sa + (sb - sa) * ((E - Ea) / (Eb - Ea));
}

}  // namespace

// ================================================================== C ABI
extern "C" {

struct oracle_config {
    double L, f, U, p, T_gas, C_meta, dt, weight, area;
    double m_e, m_OM, m_OP, M_gas;
    int32_t n_cells, ion_subcycle;
    uint32_t seed, reserved;
};

struct oracle_process {
    int32_t species, kind, target, n;
    double threshold_eV;
    const double* E_eV;
    const double* sigma_m2;
};

}  // extern "C"

namespace {

struct Proc {
    int kind, target;
    double thr;
    std::vector<double> E, s;
};

// tc = the step of the particle's next collision candidate (the end of its
// current free flight, low 32 bits of the step index).
template <class R> struct Particles {
    std::vector<R> x, vx, vy, vz;
    std::vector<uint32_t> id, tc;
    size_t size() const { return x.size(); }
    void push(R px, R pvx, R pvy, R pvz, uint32_t pid, uint32_t ptc) {
        x.push_back(px); vx.push_back(pvx); vy.push_back(pvy); vz.push_back(pvz); id.push_back(pid);
        tc.push_back(ptc);
    }
    void clear() { x.clear(); vx.clear(); vy.clear(); vz.clear(); id.clear(); tc.clear(); }
};

struct Birth4 { double x, vx, vy, vz; };

// Counter block (read by tests through oracle_counters).
struct Counters {
    uint64_t events[NSP][MAXPROC];
    uint64_t absorbed[NSP][2];     // [species][0: x<0 wall, 1: x>=L wall]
    uint64_t born[NSP];
    uint64_t neutralized;          // pairs removed by (17)
    uint64_t pair_candidates;      // pairs tested by (17)
    uint64_t particle_steps;       // particles pushed
    uint64_t warn_emax;            // energy above the table grid
    uint64_t warn_tries;           // rejection loop exhausted
    uint64_t warn_pair_gt1;        // neutralization probability > 1
    uint64_t id_overflow;
    uint64_t recombined;           // pairs removed by (16)
    uint64_t rec_candidates;       // pairs tested by (16)
    uint64_t edetached;            // pairs reacted by (22)
    uint64_t edet_candidates;      // pairs tested by (22)
    uint64_t coulomb_pairs;        // pairs scattered by (1)-(6)
    uint64_t warn_numax;           // candidates whose total rate exceeds nu_max (capped majorant)
};

template <class R> struct Oracle {
    oracle_config cfg;
    int Ng;
    double dx, n_O2, n_meta;
    double mass[NSP];
    int charge[NSP];
    // derived per-species constants in precision R
    R dt_s[NSP], qmdt[NSP], kappa[NSP], a_m[NSP], a_M[NSP], delta_el, sig_gas, sig_birth[NSP];
    R inv_dx, Lr, kappa_n, pair_factor;
    // rate tables
    std::vector<Proc> procs[NSP];
    std::vector<R> cum[NSP];          // [NGRID][nproc] cumulative rate, precision R
    std::vector<double> nu64[NSP];    // [NGRID][nproc] per-process rate, FP64
    // Conduction-current sums (Fig. 5 of the paper): for step n and species s,
    // J_sum = sum over the particles pushed in step n of trunc(256 v_x^{n+1/2})
    // (exact int64; the current density is q_s e w J_sum / (256 A L)).  On a
    // step that does not push the ions their entries repeat the last value.
    std::vector<int64_t> jhist;       // [steps since jbase][NSP]
    uint64_t jbase = 0;
    int64_t jacc[NSP] = {0, 0, 0};
    R numax[NSP], Pmax[NSP];
    double numax64[NSP];
    // majorant cap: nu_max of species s is the maximum of the total rate over
    // the grid points up to the first one at or above ecap[s] (eV); +inf =
    // the whole grid (the plain null-collision majorant)
    double ecap[NSP];
    // free flights: species s is pushed every sub[s] steps (1 for electrons,
    // the ion subcycle for ions); inv_lnq = 1 / ln(1 - P_max) = -1 / (nu_max
    // dt_s); a gap is capped at kcap pushes (2^30 steps ahead, beyond any run)
    uint32_t sub[NSP];
    R inv_lnq[NSP], kcap[NSP];
    bool tc_valid[NSP];
    bool have_neutral;
    Proc neutral;
    std::vector<R> Ktab;              // [NGRID] sigma_n g
    bool have_recomb;
    Proc recomb;
    std::vector<R> Ktab_r;            // [NGRID] sigma_r g  (16)
    R kappa_r;
    bool have_edet;
    Proc edet;
    std::vector<R> Ktab_d;            // [NGRID] sigma_22 g  (22)
    R kappa_d, thr_d;
    // Coulomb (1)-(6): enabled reactions (bit r-1 for reaction r) and, per
    // reaction, K = q_a^2 q_b^2 w lnL dt_ion / (8 pi eps0^2 mu^2 A dx) (sigma^2
    // of a pair = K N / g^3 with N the count the reaction's density uses)
    uint32_t coul_mask = 0;
    R coul_K[6], coul_fa[6], coul_fb[6];
    // state
    Particles<R> sp[NSP];
    uint64_t next_id[NSP];           // id of the next birth (64-bit: ids past 2^32 - 1 are detected)
    uint64_t step;
    std::vector<uint64_t> Q[NSP];
    std::vector<double> phi, Efield;
    std::vector<R> Eg;
    std::vector<uint64_t> Qacc[NSP];
    uint64_t acc_steps;
    Counters cnt;
    bool field_valid;
    int threads = 1;                  // host threads of the particle loop and the deposit

    explicit Oracle(const oracle_config& c) : cfg(c) {
        Ng = cfg.n_cells + 1;
        dx = cfg.L / cfg.n_cells;
        n_O2 = cfg.p / (KB * cfg.T_gas);
        n_meta = cfg.C_meta * n_O2;
        mass[SP_E] = cfg.m_e; mass[SP_OM] = cfg.m_OM; mass[SP_OP] = cfg.m_OP;
        charge[SP_E] = -1; charge[SP_OM] = -1; charge[SP_OP] = +1;
        for (int s = 0; s < NSP; ++s) {
            double dts = cfg.dt * (s == SP_E ? 1.0 : (double)cfg.ion_subcycle);
            dt_s[s] = (R)dts;
            qmdt[s] = (R)((charge[s] * QE / mass[s]) * dts);
            double mu = (s == SP_E) ? mass[s] : mass[s] * cfg.M_gas / (mass[s] + cfg.M_gas);
            kappa[s] = (R)(0.5 * mu / QE);
            a_m[s] = (R)(mass[s] / (mass[s] + cfg.M_gas));
            a_M[s] = (R)(cfg.M_gas / (mass[s] + cfg.M_gas));
            sig_birth[s] = (R)std::sqrt(KB * cfg.T_gas / mass[s]);
            numax[s] = 0; Pmax[s] = 0; numax64[s] = 0; ecap[s] = INFINITY;
            sub[s] = (s == SP_E) ? 1u : (uint32_t)cfg.ion_subcycle;
            inv_lnq[s] = (R)(-INFINITY);
            kcap[s] = (R)std::floor(1073741824.0 / (double)sub[s]);
            tc_valid[s] = false;
            Q[s].assign(Ng, 0); Qacc[s].assign(Ng, 0);
            next_id[s] = 0;
        }
        delta_el = (R)(2.0 * cfg.m_e / cfg.M_gas);
        sig_gas = (R)std::sqrt(KB * cfg.T_gas / cfg.M_gas);
        inv_dx = (R)(1.0 / dx);
        Lr = (R)cfg.L;
        double mun = cfg.m_OM * cfg.m_OP / (cfg.m_OM + cfg.m_OP);
        kappa_n = (R)(0.5 * mun / QE);
        double dt_ion = cfg.dt * (double)cfg.ion_subcycle;
        pair_factor = (R)(cfg.weight * dt_ion / (cfg.area * dx));
        const double mur = cfg.m_e * cfg.m_OP / (cfg.m_e + cfg.m_OP);
        kappa_r = (R)(0.5 * mur / QE);
        const double mud = cfg.m_e * cfg.m_OM / (cfg.m_e + cfg.m_OM);
        kappa_d = (R)(0.5 * mud / QE);
        thr_d = 0;
        have_edet = false;
        have_neutral = false;
        have_recomb = false;
        step = 0; acc_steps = 0;
        phi.assign(Ng, 0.0); Efield.assign(Ng, 0.0); Eg.assign(Ng, (R)0);
        std::memset(&cnt, 0, sizeof(cnt));
        field_valid = false;
    }

    // ---- rate tables: nu_k(E_i) = n_target sigma_k(E_i) g(E_i),
    // g = sqrt(2 e E / mu) (mu = m_e for electrons: target at rest).
    // Cumulative sums over the process order, maximum over grid points,
    // P_max = 1 - exp(-nu_max dt_s)  (null-collision method).
    int set_processes(const oracle_process* p, int n) {
        for (int s = 0; s < NSP; ++s) { procs[s].clear(); cum[s].clear(); nu64[s].clear(); }
        have_neutral = false;
        have_recomb = false;
        have_edet = false;
        for (int j = 0; j < n; ++j) {
            const oracle_process& q = p[j];
            if (q.n < 1 || q.species < 0 || q.species >= NSP) return -1;
            Proc pr; pr.kind = q.kind; pr.target = q.target; pr.thr = q.threshold_eV;
            pr.E.assign(q.E_eV, q.E_eV + q.n); pr.s.assign(q.sigma_m2, q.sigma_m2 + q.n);
            for (int i = 1; i < q.n; ++i) if (!(pr.E[i] > pr.E[i - 1])) return -1;
            if (q.kind == K_NEUTRALIZE) { neutral = pr; have_neutral = true; continue; }
            if (q.kind == K_RECOMBINE) {
                if (q.species != SP_E) return -1;
                recomb = pr; have_recomb = true; continue;
            }
            if (q.kind == K_EDETACH) {
                if (q.species != SP_OM) return -1;
                edet = pr; have_edet = true; continue;
            }
            if ((int)procs[q.species].size() >= MAXPROC) return -1;
            procs[q.species].push_back(pr);
        }
        for (int s = 0; s < NSP; ++s) {
            int np = (int)procs[s].size();
            cum[s].assign((size_t)NGRID * std::max(np, 1), (R)0);
            nu64[s].assign((size_t)NGRID * std::max(np, 1), 0.0);
            double mu = (s == SP_E) ? mass[s] : mass[s] * cfg.M_gas / (mass[s] + cfg.M_gas);
            double mx = 0.0;
            bool capped = false;      // past the first grid point at or above the cap
            for (int i = 0; i < NGRID; ++i) {
                double Ei = grid_energy(i);
                double g = std::sqrt(2.0 * QE * Ei / mu);
                double acc = 0.0;
                for (int k = 0; k < np; ++k) {
                    const Proc& pr = procs[s][k];
                    double ntar = (pr.target == T_O2_META) ? n_meta : n_O2;
                    double nu = ntar * sigma_at(pr.E, pr.s, pr.thr, Ei) * g;
                    nu64[s][(size_t)i * np + k] = nu;
                    acc += nu;
                    cum[s][(size_t)i * np + k] = (R)acc;
                }
                if (!capped) mx = std::max(mx, acc);
                if (Ei >= ecap[s]) capped = true;
            }
            numax64[s] = mx;
            numax[s] = (R)mx;
            double dts = cfg.dt * (s == SP_E ? 1.0 : (double)cfg.ion_subcycle);
            Pmax[s] = (R)(1.0 - std::exp(-mx * dts));
            inv_lnq[s] = (R)(-1.0 / (mx * dts));   // 1 / ln(1 - P_max); -inf when nu_max = 0
            tc_valid[s] = false;                  // gaps drawn with the old nu_max: draw afresh
        }
        Ktab.assign(NGRID, (R)0);
        if (have_neutral) {
            double mun = cfg.m_OM * cfg.m_OP / (cfg.m_OM + cfg.m_OP);
            for (int i = 0; i < NGRID; ++i) {
                double Ei = grid_energy(i);
                double g = std::sqrt(2.0 * QE * Ei / mun);
                Ktab[i] = (R)(sigma_at(neutral.E, neutral.s, neutral.thr, Ei) * g);
            }
        }
        // (22): sigma g with the e-O- reduced mass; the threshold (O's
        // electron affinity) also bounds the reaction (see pair_process)
        Ktab_d.assign(NGRID, (R)0);
        thr_d = have_edet ? (R)edet.thr : (R)0;
        if (have_edet) {
            double mud = cfg.m_e * cfg.m_OM / (cfg.m_e + cfg.m_OM);
            for (int i = 0; i < NGRID; ++i) {
                double Ei = grid_energy(i);
                double g = std::sqrt(2.0 * QE * Ei / mud);
                Ktab_d[i] = (R)(sigma_at(edet.E, edet.s, edet.thr, Ei) * g);
            }
        }
        Ktab_r.assign(NGRID, (R)0);
        if (have_recomb) {
            double mur = cfg.m_e * cfg.m_OP / (cfg.m_e + cfg.m_OP);
            for (int i = 0; i < NGRID; ++i) {
                double Ei = grid_energy(i);
                double g = std::sqrt(2.0 * QE * Ei / mur);
                Ktab_r[i] = (R)(sigma_at(recomb.E, recomb.s, recomb.thr, Ei) * g);
            }
        }
        return 0;
    }

    // ---- CIC weights, fixed point: r = trunc(frac * 2^16); node j gets
    // 2^16 - r, node j+1 gets r (sum exactly 2^16 per particle).
    void cell_of(R x, int& j, R& frac) const {
        R s = x * inv_dx;
        j = (int)s;
        if (j > cfg.n_cells - 1) j = cfg.n_cells - 1;
        frac = s - (R)j;
    }
    void deposit_one(std::vector<uint64_t>& q, R x) const {
        int j; R frac; cell_of(x, j, frac);
        uint32_t r = (uint32_t)(frac * (R)FIX_ONE);
        q[j] += (uint64_t)(65536u - r);
        q[j + 1] += (uint64_t)r;
    }
    void deposit_all() {
        for (int s = 0; s < NSP; ++s) {
            std::fill(Q[s].begin(), Q[s].end(), 0);
            const long long N = (long long)sp[s].size();
            int T = std::max(1, threads);
            if ((long long)T > N / 4096 + 1) T = (int)(N / 4096 + 1);
            // integer sums: per-thread arrays added in any order give the same Q
            std::vector<std::vector<uint64_t>> tq(T, std::vector<uint64_t>(Ng, 0));
#pragma omp parallel for schedule(static) num_threads(T)
            for (long long i = 0; i < N; ++i) {
#ifdef _OPENMP
                const int t = omp_get_thread_num();
#else
                const int t = 0;
#endif
                deposit_one(tq[t], sp[s].x[i]);
            }
            for (int t = 0; t < T; ++t)
                for (int j = 0; j < Ng; ++j) Q[s][j] += tq[t][j];
        }
    }

    // ---- Poisson (FP64): interior nodes j = 1..N-1,
    //   -phi_{j-1} + 2 phi_j - phi_{j+1} = rho_j dx^2 / eps0,
    // phi_0 = U sin(2 pi f t) (driven electrode at x = 0), phi_N = 0 (grounded).
    void field_solve(double t) {
        int N = cfg.n_cells;
        std::vector<long long> Rn(Ng);
        for (int j = 0; j < Ng; ++j)
            Rn[j] = (long long)Q[SP_OP][j] - (long long)Q[SP_E][j] - (long long)Q[SP_OM][j];
        double V0 = cfg.U * std::sin(TWO_PI * cfg.f * t);
        solve_field(N, dx, cfg.weight, cfg.area, V0, Rn.data(), phi.data(), Efield.data());
        for (int j = 0; j < Ng; ++j) Eg[j] = (R)Efield[j];
        field_valid = true;
    }

    // Poisson (Sec. 2), Dirichlet at both walls.  With the net node charge R_j
    // (2^16 units per macro-particle) the interior equations read
    //   (phi_{j+1} - phi_j) - (phi_j - phi_{j-1}) = -c R_j,
    //   c = e w dx / (A eps0 2^16),
    // i.e. a discrete double integration: with S_m = sum_{k=1..m} R_k and
    // T_j = sum_{m<j} S_m (exact integers), D_0 = phi_1 - phi_0 follows from
    // phi_N = 0 and
    //   phi_j = V0 + j D_0 - c T_j,   D_j = phi_{j+1} - phi_j = D_0 - c S_j.
    // E = -dphi/dx by central differences inside, E_j = -(D_j + D_{j-1})/(2dx);
    // at the walls from Gauss's law over the half cell, E_0 = (-D_0 - c R_0)/dx,
    // E_N = (-D_{N-1} + c R_N)/dx.  This is the exact solution of the same
    // tridiagonal system the Thomas algorithm solves (solve_field_thomas,
    // kept to pin it); the only rounding is in the final FP64 expressions.
    static void solve_field(int N, double dx, double w, double A, double V0, const long long* Rn,
                            double* phi, double* E) {
        const double c = QE * w * dx / (A * EPS0 * FIX_ONE);
        std::vector<long long> S(N + 1, 0), T(N + 1, 0);
        for (int m = 1; m <= N; ++m) S[m] = S[m - 1] + Rn[m];
        for (int j = 1; j <= N; ++j) T[j] = T[j - 1] + S[j - 1];
        const double D0 = (c * (double)T[N] - V0) / (double)N;
        for (int j = 0; j <= N; ++j) {
            if (j == 0) phi[j] = V0;
            else if (j == N) phi[j] = 0.0;
            else phi[j] = V0 + (double)j * D0 - c * (double)T[j];
        }
        const double inv_dx = 1.0 / dx, inv_2dx = 1.0 / (2.0 * dx);
        for (int j = 1; j <= N - 1; ++j) E[j] = (c * (double)(S[j] + S[j - 1]) - 2.0 * D0) * inv_2dx;
        E[0] = (-D0 - c * (double)Rn[0]) * inv_dx;
        E[N] = (c * (double)S[N - 1] - D0 + c * (double)Rn[N]) * inv_dx;
    }

    // The same system by the Thomas algorithm (a = c = -1, b = 2) with the
    // boundary values moved to the right-hand side; E as above.  Test use.
    static void solve_field_thomas(int N, double dx, double w, double A, double V0, const long long* Rn,
                                   double* phi, double* E) {
        std::vector<double> rhs(N + 1, 0.0), cp(N + 1, 0.0), dp(N + 1, 0.0);
        for (int j = 1; j <= N - 1; ++j) {
            double rho = QE * w * (double)Rn[j] / (FIX_ONE * A * dx);
            rhs[j] = rho * dx * dx / EPS0;
        }
        phi[0] = V0; phi[N] = 0.0;
        if (N >= 2) {
            rhs[1] += V0;
            cp[1] = -1.0 / 2.0;
            dp[1] = rhs[1] / 2.0;
            for (int j = 2; j <= N - 1; ++j) {
                double den = 2.0 + cp[j - 1];
                cp[j] = -1.0 / den;
                dp[j] = (rhs[j] + dp[j - 1]) / den;
            }
            phi[N - 1] = dp[N - 1];
            for (int j = N - 2; j >= 1; --j) phi[j] = dp[j] - cp[j] * phi[j + 1];
        }
        for (int j = 1; j <= N - 1; ++j) E[j] = (phi[j - 1] - phi[j + 1]) / (2.0 * dx);
        double q0 = QE * w * (double)Rn[0] / FIX_ONE;
        double qN = QE * w * (double)Rn[N] / FIX_ONE;
        E[0] = (phi[0] - phi[1]) / dx - q0 / (EPS0 * A);
        E[N] = (phi[N - 1] - phi[N]) / dx + qN / (EPS0 * A);
    }

    // ---- free flights (Sec. 2: "the durations of the free flights ... from
    // elementary kinetic considerations").  In the null-collision method a
    // particle's candidate collisions form a Poisson process of rate nu_max;
    // on the time grid of its pushes (every sub[s] steps of dt) the number K
    // of pushes without a candidate is geometric,
    // P(K >= k) = exp(-k nu_max dt_s) = (1 - P_max)^k, drawn by inversion as
    // K = floor(ln(u) / ln(1 - P_max)) with u = ((w >> 8) + 1/2) 2^-24 in (0, 1).
    // This is the same law as a Bernoulli(P_max) test at every push.
    uint32_t flight_gap(int s, uint32_t w) const {
        const R u = ((R)(w >> 8) + (R)0.5) * (R)(1.0 / 16777216.0);
        const R t = ln_(u) * inv_lnq[s];
        const R k = std::floor(t);
        return (k < kcap[s]) ? (uint32_t)k : (uint32_t)kcap[s];
    }
    // The first step >= n at which species s is pushed.
    uint64_t first_push(int s, uint64_t n) const {
        return (n + sub[s] - 1) / sub[s] * sub[s];
    }
    // A fresh free flight for particle `id` of species s whose first push is
    // at step nf, drawn from its stream at step n with tag TAG_FLIGHT + s.
    uint32_t fresh_tc(int s, uint32_t id, uint64_t n, uint64_t nf) const {
        const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(TAG_FLIGHT + s), 0u, (uint32_t)(n >> 32)};
        const uint32_t key[2] = {id, cfg.seed};
        const U4 w = philox4x32_10(ctr, key);
        return (uint32_t)(nf + (uint64_t)sub[s] * flight_gap(s, w.v[0]));
    }
    // Free flights of the loaded particles of every species whose flights are
    // not known (after a load or new tables), drawn at step n.
    void draw_flights(uint64_t n) {
        for (int s = 0; s < NSP; ++s) {
            if (tc_valid[s]) continue;
            const uint64_t nf = first_push(s, n);
            for (size_t i = 0; i < sp[s].size(); ++i) sp[s].tc[i] = fresh_tc(s, sp[s].id[i], n, nf);
            tc_valid[s] = true;
        }
    }

    // ---- table lookups
    R cum_at(int s, int k, int i, R w) const {
        return grid_interp<R>(cum[s], (int)procs[s].size(), k, i, w);
    }

    // ---- one particle: push, absorb, null-collision MCC.
    // Returns false if the particle leaves the arrays (absorbed or consumed).
    // Births are appended to `births[dst]` in generation order.

    bool update_particle(int s, uint64_t n, R& x, R& vx, R& vy, R& vz, uint32_t id, uint32_t& tc,
                         std::vector<Birth4>* births, const std::vector<R>& Ef) {
        return update_particle(s, n, x, vx, vy, vz, id, tc, births, Ef, cnt, jacc[s]);
    }
    bool update_particle(int s, uint64_t n, R& x, R& vx, R& vy, R& vz, uint32_t id, uint32_t& tc,
                         std::vector<Birth4>* births, const std::vector<R>& Ef, Counters& cnt, int64_t& jsum) {
        // gather: E_p = E_j + frac (E_{j+1} - E_j)
        int j; R frac; cell_of(x, j, frac);
        R Ep = fma_(frac, Ef[j + 1] - Ef[j], Ef[j]);
        // leapfrog: v^{n+1/2} = v^{n-1/2} + (q/m) E dt ; x^{n+1} = x^n + v^{n+1/2} dt
        vx = fma_(qmdt[s], Ep, vx);
        x = fma_(vx, dt_s[s], x);
        cnt.particle_steps += 1;
        jsum += (int64_t)(vx * (R)256);      // exact scaling by 2^8, then truncation
        // absorbing electrodes
        if (x < (R)0) { cnt.absorbed[s][0] += 1; return false; }
        if (x >= Lr) { cnt.absorbed[s][1] += 1; return false; }
        return collide(s, n, x, vx, vy, vz, id, tc, births, cnt);
    }

    bool collide(int s, uint64_t n, R x, R& vx, R& vy, R& vz, uint32_t id, uint32_t& tc,
                 std::vector<Birth4>* births, Counters& cnt) {
        int np = (int)procs[s].size();
        if (np == 0) return true;
        if (tc != (uint32_t)n) return true;        // in free flight: no candidate this step
        // a candidate: word 0 of the step's stream draws the next free flight,
        // word 1 the real/null test, the rest the kinematics
        Stream st(id, cfg.seed, n, (uint32_t)(s == SP_E ? TAG_E : (s == SP_OM ? TAG_OM : TAG_OP)));
        tc = (uint32_t)(n + (uint64_t)sub[s] * (1u + (uint64_t)flight_gap(s, st.next())));
        R u1 = uniform<R>(st.next());
        uint64_t& warn = cnt.warn_tries;
        R vt[3] = {0, 0, 0};
        R E, gx = vx, gy = vy, gz = vz;
        if (s != SP_E) {
            maxwellian<R>(st, sig_gas, vt, warn);  // O2 target at T_gas
            gx = vx - vt[0]; gy = vy - vt[1]; gz = vz - vt[2];
        }
        E = kappa[s] * dot3<R>(gx, gy, gz, gx, gy, gz);
        int i; R w; bool above;
        grid_locate<R>(E, i, w, above);
        if (above) cnt.warn_emax += 1;
        // null-collision method: the candidate is a null collision unless
        // u1 nu_max falls below the total rate nu(E); the process is then the
        // first k with u1 nu_max < sum_{i<=k} nu_i(E) (the last process if
        // rounding leaves none below it)
        R target = u1 * numax[s];
        const R total = cum_at(s, np - 1, i, w);
        if (total > numax[s]) cnt.warn_numax += 1;   // above a capped majorant
        if (!(target < total)) return true;   // null collision
        int k = np - 1;
        for (int kk = 0; kk < np - 1; ++kk) {
            if (target < cum_at(s, kk, i, w)) { k = kk; break; }
        }
        const Proc& pr = procs[s][k];
        if (E < (R)pr.thr) return true;             // below threshold: null
        cnt.events[s][k] += 1;
        switch (pr.kind) {
        case K_ELASTIC: {
            R nh[3]; isotropic<R>(st, nh, warn);
            if (s == SP_E) {
                // isotropic scattering off a heavy target at rest:
                // |v'|^2 = |v|^2 (1 - (2 m/M)(1 - cos chi))
                R v2 = dot3<R>(vx, vy, vz, vx, vy, vz);
                R vm = sqrt_(v2);
                R cosx = (vm > (R)0) ? dot3<R>(nh[0], nh[1], nh[2], vx, vy, vz) / vm : (R)0;
                R fac = (R)1 - delta_el * ((R)1 - cosx);
                R vn = vm * sqrt_(fac);
                vx = vn * nh[0]; vy = vn * nh[1]; vz = vn * nh[2];
            } else {
                // isotropic in the centre-of-mass frame
                R gm = sqrt_(dot3<R>(gx, gy, gz, gx, gy, gz));
                R cmx = fma_(a_m[s], vx, a_M[s] * vt[0]);
                R cmy = fma_(a_m[s], vy, a_M[s] * vt[1]);
                R cmz = fma_(a_m[s], vz, a_M[s] * vt[2]);
                R f = a_M[s] * gm;
                vx = fma_(f, nh[0], cmx); vy = fma_(f, nh[1], cmy); vz = fma_(f, nh[2], cmz);
            }
            return true;
        }
        case K_EXCITE: {
            R Ep = E - (R)pr.thr;
            R nh[3]; isotropic<R>(st, nh, warn);
            R vn = sqrt_(Ep / kappa[s]);
            vx = vn * nh[0]; vy = vn * nh[1]; vz = vn * nh[2];
            return true;
        }
        case K_IONIZE: {
            R Er = E - (R)pr.thr;
            R u = uniform<R>(st.next());
            R Es = u * Er;
            R Epr = Er - Es;
            R n1[3], n2[3], vi[3];
            isotropic<R>(st, n1, warn);
            isotropic<R>(st, n2, warn);
            maxwellian<R>(st, sig_birth[SP_OP], vi, warn);
            R vp = sqrt_(Epr / kappa[SP_E]);
            R vs = sqrt_(Es / kappa[SP_E]);
            vx = vp * n1[0]; vy = vp * n1[1]; vz = vp * n1[2];
            births[SP_E].push_back({(double)x, (double)(vs * n2[0]), (double)(vs * n2[1]), (double)(vs * n2[2])});
            births[SP_OP].push_back({(double)x, (double)vi[0], (double)vi[1], (double)vi[2]});
            return true;
        }
        case K_ATTACH: {
            R vi[3]; maxwellian<R>(st, sig_birth[SP_OM], vi, warn);
            births[SP_OM].push_back({(double)x, (double)vi[0], (double)vi[1], (double)vi[2]});
            return false;
        }
        case K_DETACH: {
            R Er = E - (R)pr.thr;
            R nh[3]; isotropic<R>(st, nh, warn);
            R vn = sqrt_(Er / kappa[SP_E]);
            births[SP_E].push_back({(double)x, (double)(vn * nh[0]), (double)(vn * nh[1]), (double)(vn * nh[2])});
            return false;
        }
        case K_CX: {
            vx = vt[0]; vy = vt[1]; vz = vt[2];
            return true;
        }
        default:
            return true;
        }
    }

    void process_species(int s, uint64_t n, std::vector<Birth4>* births) {
        Particles<R>& P = sp[s];
        const long long N = (long long)P.size();
        int T = std::max(1, threads);
        if ((long long)T > N / 4096 + 1) T = (int)(N / 4096 + 1);
        // thread t takes the t-th contiguous range (schedule(static)); its
        // counters, current sum and births are merged below in range order
        std::vector<Counters> tcnt(T);
        std::vector<int64_t> tj(T, 0);
        std::vector<std::vector<Birth4>> tb((size_t)T * NSP);
        for (Counters& c : tcnt) std::memset(&c, 0, sizeof(c));
        std::vector<char> alive((size_t)N);
#pragma omp parallel for schedule(static) num_threads(T)
        for (long long i = 0; i < N; ++i) {
#ifdef _OPENMP
            const int t = omp_get_thread_num();
#else
            const int t = 0;
#endif
            R x = P.x[i], vx = P.vx[i], vy = P.vy[i], vz = P.vz[i];
            uint32_t tc = P.tc[i];
            alive[i] = update_particle(s, n, x, vx, vy, vz, P.id[i], tc, &tb[(size_t)t * NSP], Eg, tcnt[t], tj[t])
                           ? 1 : 0;
            P.x[i] = x; P.vx[i] = vx; P.vy[i] = vy; P.vz[i] = vz; P.tc[i] = tc;
        }
        for (int t = 0; t < T; ++t) {
            const uint64_t* a = reinterpret_cast<const uint64_t*>(&tcnt[t]);
            uint64_t* b = reinterpret_cast<uint64_t*>(&cnt);
            for (size_t k = 0; k < sizeof(Counters) / sizeof(uint64_t); ++k) b[k] += a[k];
            jacc[s] += tj[t];
            for (int d = 0; d < NSP; ++d)
                births[d].insert(births[d].end(), tb[(size_t)t * NSP + d].begin(), tb[(size_t)t * NSP + d].end());
        }
        filter(P, alive, true);
    }

    // ---- cell-binned binary processes between species A and B (the
    // reading of (17), also used for (16)).  In each cell j, list the A and
    // the B particles in array order; with m = min(nA, nB), M = max(nA, nB)
    // and a cell shift r_j drawn per cell and step, the i-th member of the
    // shorter list (i < m) is paired with member (i + r_j) mod M of the
    // longer list (A counts as shorter on a tie).  A pair reacts with
    // probability P = M w sigma(E_rel) g dt_ion / (A dx), which gives
    // nA nB w <sigma g> dt / (A dx) reactions per cell and step; both
    // particles are removed.  The acceptance number comes from the A
    // particle's stream.
    // mode 0: both particles of a reacted pair are removed ((16), (17));
    // mode 1, (22) e + O- -> O + 2e with A = O-, B = e: a pair reacts only at
    // or above the threshold thr; the O- is removed, the electron loses thr,
    // the rest E - thr is split uniformly between it and the detached electron
    // (fraction from the O-'s stream after its acceptance number), both going
    // off isotropically from the O-'s velocity; the newborn, at the O-'s
    // position, goes to births22 keyed by the O-'s array index.
    void pair_process(uint64_t n, int A, int B, const std::vector<R>& K_tab, R kap, uint32_t tag_shift,
                      uint32_t tag_pair, uint64_t& tested, uint64_t& reacted, int mode = 0, R thr = (R)0,
                      std::vector<std::pair<size_t, Birth4>>* births22 = nullptr) {
        int Nc = cfg.n_cells;
        std::vector<std::vector<size_t>> LA(Nc), LB(Nc);
        for (size_t i = 0; i < sp[A].size(); ++i) { int j; R fr; cell_of(sp[A].x[i], j, fr); LA[j].push_back(i); }
        for (size_t i = 0; i < sp[B].size(); ++i) { int j; R fr; cell_of(sp[B].x[i], j, fr); LB[j].push_back(i); }
        std::vector<char> deadA(sp[A].size(), 0), deadB(sp[B].size(), 0);
        for (int c = 0; c < Nc; ++c) {
            size_t na = LA[c].size(), nb = LB[c].size();
            size_t m = std::min(na, nb), M = std::max(na, nb);
            if (m == 0) continue;
            Stream sh((uint32_t)c, cfg.seed, n, tag_shift);
            uint32_t r = (uint32_t)(sh.next() % (uint32_t)M);
            bool a_short = (na <= nb);
            for (size_t i = 0; i < m; ++i) {
                size_t partner = (i + r) % M;
                size_t a = a_short ? LA[c][i] : LA[c][partner];
                size_t b = a_short ? LB[c][partner] : LB[c][i];
                Stream st(sp[A].id[a], cfg.seed, n, tag_pair);
                R u = uniform<R>(st.next());
                R gx = sp[A].vx[a] - sp[B].vx[b];
                R gy = sp[A].vy[a] - sp[B].vy[b];
                R gz = sp[A].vz[a] - sp[B].vz[b];
                R E = kap * dot3<R>(gx, gy, gz, gx, gy, gz);
                int gi; R gw; bool above;
                grid_locate<R>(E, gi, gw, above);
                if (above) cnt.warn_emax += 1;
                R K = grid_interp<R>(K_tab, 1, 0, gi, gw);
                R P = K * (pair_factor * (R)M);
                tested += 1;
                if (P > (R)1) cnt.warn_pair_gt1 += 1;
                if (!(u < P) || E < thr) continue;
                reacted += 1;
                deadA[a] = 1;
                if (mode == 0) { deadB[b] = 1; continue; }
                const R Er = E - thr;
                const R us = uniform<R>(st.next());
                const R Es = us * Er;
                const R Ep = Er - Es;
                R n1[3], n2[3];
                isotropic<R>(st, n1, cnt.warn_tries);
                isotropic<R>(st, n2, cnt.warn_tries);
                const R vp = sqrt_(Ep / kappa[SP_E]);
                const R vs = sqrt_(Es / kappa[SP_E]);
                const R ax = sp[A].vx[a], ay = sp[A].vy[a], az = sp[A].vz[a];
                sp[B].vx[b] = ax + vp * n1[0];
                sp[B].vy[b] = ay + vp * n1[1];
                sp[B].vz[b] = az + vp * n1[2];
                births22->push_back({a, {(double)sp[A].x[a], (double)(ax + vs * n2[0]), (double)(ay + vs * n2[1]),
                                         (double)(az + vs * n2[2])}});
            }
        }
        filter(sp[A], deadA);
        filter(sp[B], deadB);
    }

    // (17) O- + O2+ -> O + O2
    void neutralize(uint64_t n) {
        if (!have_neutral) return;
        pair_process(n, SP_OM, SP_OP, Ktab, kappa_n, TAG_SHIFT, TAG_PAIR, cnt.pair_candidates, cnt.neutralized);
    }

    // ---- Coulomb elastic collisions (1)-(6) of Table 1, by the binary
    // collision model of Takizuka & Abe (J. Comput. Phys. 25, 205, 1977):
    // within a cell each pair's relative velocity u (|u| = g) turns by an angle
    // theta with tan(theta/2) = delta ~ N(0, sigma^2), sigma^2 = K N / g^3, and
    // an azimuth phi uniform on [0, 2 pi); momentum and energy of the pair are
    // kept.  Readings: on ion steps with dt_ion, after the species' pushes and
    // before the reactive pairs, reactions in the order (1)..(6); pairs from
    // the cell lists in array order: like species by a random rotation r of
    // the list, (q_r, q_r+1), (q_r+2, q_r+3), ... (an odd one sits out), N =
    // the species' count in the cell; unlike species the i-th of the shorter
    // list with member (i + r) mod M of the longer (as (17)), N = M, the
    // larger count (each member of the longer list then collides with
    // probability m/M, with that much larger a variance, so that both species
    // get the model's mean-square deflection rate).  delta from the first
    // member's stream (tag 12 + reaction index): one polar normal, then phi
    // as the double angle of a uniform point of the unit disk.
    void coulomb_pair(int r, int a, size_t ia, int b, size_t ib, R N, uint64_t n, Counters& c) {
        R& ax = sp[a].vx[ia]; R& ay = sp[a].vy[ia]; R& az = sp[a].vz[ia];
        R& bx = sp[b].vx[ib]; R& by = sp[b].vy[ib]; R& bz = sp[b].vz[ib];
        const R ux = ax - bx, uy = ay - by, uz = az - bz;
        const R g2 = dot3<R>(ux, uy, uz, ux, uy, uz);
        if (!(g2 > (R)0)) return;
        const R g = sqrt_(g2);
        Stream st(sp[a].id[ia], cfg.seed, n, (uint32_t)(TAG_COUL + r));
        R z0, z1;
        normal_pair<R>(st, z0, z1, c.warn_tries);
        const R sig2 = coul_K[r] * N / (g2 * g);
        const R d = sqrt_(sig2) * z0;
        R sn, omc;   // sin(theta), 1 - cos(theta)
        if (std::fabs(d) < (R)1e18) {
            const R q = (R)1 / ((R)1 + d * d);
            sn = (R)2 * d * q;
            omc = (R)2 * (d * d) * q;
        } else {
            sn = (R)0; omc = (R)2;
        }
        R cp = (R)1, spn = (R)0;   // cos(phi), sin(phi)
        for (int t = 0; t < MAX_TRIES; ++t) {
            const R e1 = (R)2 * uniform<R>(st.next()) - (R)1;
            const R e2 = (R)2 * uniform<R>(st.next()) - (R)1;
            const R s2 = e1 * e1 + e2 * e2;
            if (s2 > (R)0 && s2 < (R)1) { cp = (e1 * e1 - e2 * e2) / s2; spn = ((R)2 * e1 * e2) / s2; break; }
            if (t == MAX_TRIES - 1) c.warn_tries += 1;
        }
        const R up2 = ux * ux + uy * uy;
        R dx, dy, dz;
        if (up2 > (R)0) {
            const R up = sqrt_(up2);
            const R sc = sn * cp, ss = sn * spn;
            dx = (ux * uz / up) * sc - (uy * g / up) * ss - ux * omc;
            dy = (uy * uz / up) * sc + (ux * g / up) * ss - uy * omc;
            dz = -up * sc - uz * omc;
        } else {
            dx = g * (sn * cp);
            dy = g * (sn * spn);
            dz = -uz * omc;
        }
        ax = ax + coul_fa[r] * dx; ay = ay + coul_fa[r] * dy; az = az + coul_fa[r] * dz;
        bx = bx - coul_fb[r] * dx; by = by - coul_fb[r] * dy; bz = bz - coul_fb[r] * dz;
        c.coulomb_pairs += 1;
    }

    void set_coulomb(uint32_t mask, double ln_lambda) {
        coul_mask = mask & 63u;
        const double mass[NSP] = {cfg.m_e, cfg.m_OM, cfg.m_OP};
        const double dx = cfg.L / cfg.n_cells, dti = cfg.dt * (double)cfg.ion_subcycle;
        const double q4 = QE * QE * QE * QE;
        for (int r = 0; r < 6; ++r) {
            const double ma = mass[COUL_PAIRS[r][0]], mb = mass[COUL_PAIRS[r][1]];
            const double mu = ma * mb / (ma + mb);
            coul_K[r] = (R)(q4 * cfg.weight * ln_lambda * dti / (8.0 * M_PI * EPS0 * EPS0 * mu * mu * cfg.area * dx));
            coul_fa[r] = (R)(mb / (ma + mb));
            coul_fb[r] = (R)(ma / (ma + mb));
        }
    }

    void coulomb(uint64_t n) {
        if (!coul_mask) return;
        const int Nc = cfg.n_cells;
        for (int r = 0; r < 6; ++r) {
            if (!((coul_mask >> r) & 1u)) continue;
            const int a = COUL_PAIRS[r][0], b = COUL_PAIRS[r][1];
            std::vector<std::vector<size_t>> LA(Nc), LB(Nc);
            for (size_t i = 0; i < sp[a].size(); ++i) { int j; R fr; cell_of(sp[a].x[i], j, fr); LA[j].push_back(i); }
            if (a != b)
                for (size_t i = 0; i < sp[b].size(); ++i) { int j; R fr; cell_of(sp[b].x[i], j, fr); LB[j].push_back(i); }
            for (int c = 0; c < Nc; ++c) {
                const size_t na = LA[c].size(), nb = (a == b) ? na : LB[c].size();
                if (a == b ? na < 2 : (na == 0 || nb == 0)) continue;
                const size_t M = std::max(na, nb), m = std::min(na, nb);
                Stream sh((uint32_t)c, cfg.seed, n, (uint32_t)(TAG_SHIFT_COUL + r));
                const size_t rs = (size_t)(sh.next() % (uint32_t)M);
                if (a == b) {
                    for (size_t j = 0; 2 * j + 1 < na; ++j)
                        coulomb_pair(r, a, LA[c][(rs + 2 * j) % na], a, LA[c][(rs + 2 * j + 1) % na], (R)na, n, cnt);
                } else {
                    const bool a_short = na <= nb;
                    for (size_t i = 0; i < m; ++i) {
                        const size_t p = (i + rs) % M;
                        coulomb_pair(r, a, a_short ? LA[c][i] : LA[c][p], b, a_short ? LB[c][p] : LB[c][i], (R)M, n,
                                     cnt);
                    }
                }
            }
        }
    }

    // (22) e + O- -> O + 2e, on ion steps before (16) and (17) (reading: the
    // paper gives no order); its births follow the step's other electron
    // births, in the order of their O- parents.
    void edetach(uint64_t n, std::vector<Birth4>* births) {
        if (!have_edet) return;
        std::vector<std::pair<size_t, Birth4>> b22;
        pair_process(n, SP_OM, SP_E, Ktab_d, kappa_d, TAG_SHIFT_EDET, TAG_EDET, cnt.edet_candidates, cnt.edetached,
                     1, thr_d, &b22);
        std::sort(b22.begin(), b22.end(), [](const std::pair<size_t, Birth4>& p, const std::pair<size_t, Birth4>& q) {
            return p.first < q.first;
        });
        for (const auto& e : b22) births[SP_E].push_back(e.second);
    }

    // (16) e + O2+ -> O + O, on ion steps before (17) (reading: the paper
    // gives no order; the two then never claim the same O2+)
    void recombine(uint64_t n) {
        if (!have_recomb) return;
        pair_process(n, SP_E, SP_OP, Ktab_r, kappa_r, TAG_SHIFT_REC, TAG_REC, cnt.rec_candidates, cnt.recombined);
    }

    // Keep the particles not marked dead (or, keep_marked: those marked), in order.
    static void filter(Particles<R>& P, const std::vector<char>& mark, bool keep_marked = false) {
        Particles<R> out;
        for (size_t i = 0; i < P.size(); ++i)
            if ((mark[i] != 0) == keep_marked) out.push(P.x[i], P.vx[i], P.vy[i], P.vz[i], P.id[i], P.tc[i]);
        P = out;
    }

    // Births of step n take ids next_id, next_id + 1, ... in canonical order.
    // Ids are 32-bit: a birth whose id would be 2^32 or more is an id overflow
    // (counted per birth; the particle keeps the low 32 bits of its id).  A
    // newborn starts a free flight at its first push after step n.
    void append_births(std::vector<Birth4>* births, uint64_t n) {
        for (int s = 0; s < NSP; ++s) {
            const uint64_t nf = first_push(s, n + 1);
            for (const Birth4& b : births[s]) {
                const uint64_t id64 = next_id[s]++;
                if (id64 > 0xFFFFFFFFull) cnt.id_overflow += 1;
                const uint32_t id = (uint32_t)id64;
                sp[s].push((R)b.x, (R)b.vx, (R)b.vy, (R)b.vz, id, fresh_tc(s, id, n, nf));
                cnt.born[s] += 1;
            }
        }
    }

    void ensure_field() {
        if (!field_valid) { deposit_all(); field_solve((double)step * cfg.dt); }
    }

    // ---- one time step n -> n+1.
    void do_step() {
        ensure_field();
        uint64_t n = step;
        draw_flights(n);
        bool ion_step = (n % (uint64_t)cfg.ion_subcycle) == 0;
        std::vector<Birth4> births[NSP];
        for (int s = 0; s < NSP; ++s) jacc[s] = 0;
        process_species(SP_E, n, births);
        if (ion_step) {
            process_species(SP_OM, n, births);
            process_species(SP_OP, n, births);
            coulomb(n);
            edetach(n, births);
            recombine(n);
            neutralize(n);
        }
        append_births(births, n);
        deposit_all();
        field_solve((double)(n + 1) * cfg.dt);
        for (int s = 0; s < NSP; ++s)
            for (int j = 0; j < Ng; ++j) Qacc[s][j] += Q[s][j];
        acc_steps += 1;
        if (jhist.empty()) jbase = n;
        const size_t prev = jhist.size();
        for (int s = 0; s < NSP; ++s) {
            const bool pushed = (s == SP_E) || ion_step;
            jhist.push_back(pushed ? jacc[s] : (prev ? jhist[prev - NSP + s] : 0));
        }
        step = n + 1;
    }
};

struct Handle {
    int precision;   // 32 or 64
    Oracle<float>* f;
    Oracle<double>* d;
};


// One particle through push + absorb + MCC with a given gather field.
template <class R>
int update_one(Oracle<R>& O, int s, uint64_t n, const double* Ef, double* state, uint32_t id, uint32_t* tc,
               int fresh, double* births, int* nb) {
    if (fresh) *tc = O.fresh_tc(s, id, n, O.first_push(s, n));
    std::vector<R> Eg(O.Ng);
    for (int j = 0; j < O.Ng; ++j) Eg[j] = (R)Ef[j];
    R x = (R)state[0], vx = (R)state[1], vy = (R)state[2], vz = (R)state[3];
    std::vector<Birth4> b[NSP];
    int alive = O.update_particle(s, n, x, vx, vy, vz, id, *tc, b, Eg) ? 1 : 0;
    state[0] = x; state[1] = vx; state[2] = vy; state[3] = vz;
    int k = 0;
    for (int d = 0; d < NSP; ++d)
        for (const Birth4& bb : b[d]) {
            births[5 * k + 0] = d; births[5 * k + 1] = bb.x; births[5 * k + 2] = bb.vx;
            births[5 * k + 3] = bb.vy; births[5 * k + 4] = bb.vz; ++k;
        }
    *nb = k;
    return alive;
}

}  // namespace

// ================================================================== exports
extern "C" {

void* oracle_create(const oracle_config* cfg, int precision) {
    if (!cfg || cfg->n_cells < 1 || cfg->ion_subcycle < 1 || !(cfg->L > 0) || !(cfg->dt > 0)) return nullptr;
    Handle* h = new Handle();
    h->precision = precision;
    h->f = nullptr; h->d = nullptr;
    if (precision == 64) h->d = new Oracle<double>(*cfg);
    else h->f = new Oracle<float>(*cfg);
    return h;
}

void oracle_destroy(void* p) {
    Handle* h = (Handle*)p;
    if (!h) return;
    delete h->f; delete h->d; delete h;
}

#define DISPATCH(h, expr) do { if ((h)->f) { auto& O = *(h)->f; expr; } else { auto& O = *(h)->d; expr; } } while (0)

int oracle_set_processes(void* p, const oracle_process* procs, int n) {
    Handle* h = (Handle*)p; int rc = 0;
    DISPATCH(h, rc = O.set_processes(procs, n));
    return rc;
}

// Majorant caps (eV) per species, taking effect at the next
// oracle_set_processes: nu_max = the largest total rate over the grid points
// up to the first one at or above the cap (+inf or NaN: the whole grid).
// Returns -1 for a cap that is not positive.
int oracle_set_majorant_cap(void* p, const double* cap) {
    Handle* h = (Handle*)p;
    for (int s = 0; s < NSP; ++s) if (!(cap[s] > 0) && !std::isnan(cap[s])) return -1;
    DISPATCH(h, for (int s = 0; s < NSP; ++s) O.ecap[s] = std::isnan(cap[s]) ? INFINITY : cap[s]);
    return 0;
}

int oracle_load(void* p, int s, const float* x, const float* vx, const float* vy, const float* vz,
                const uint32_t* id, uint64_t n) {
    Handle* h = (Handle*)p;
    if (s < 0 || s >= NSP) return -1;
    DISPATCH(h, {
        O.sp[s].clear();
        uint64_t mx = 0;
        for (uint64_t i = 0; i < n; ++i) {
            O.sp[s].push(x[i], vx[i], vy[i], vz[i], id[i], 0u);
            mx = std::max<uint64_t>(mx, (uint64_t)id[i] + 1u);
        }
        O.tc_valid[s] = false;   // free flights drawn at the next step
        O.next_id[s] = mx;
        O.field_valid = false;
        O.jhist.clear();
    });
    return 0;
}

// Free flights of species s (the step of each particle's next collision
// candidate, in array order) after a load: n must be the particle count.
int oracle_load_flight(void* p, int s, const uint32_t* tc, uint64_t n) {
    Handle* h = (Handle*)p; int rc = 0;
    DISPATCH(h, {
        if (n != O.sp[s].size()) rc = -1;
        else { for (uint64_t i = 0; i < n; ++i) O.sp[s].tc[i] = tc[i]; O.tc_valid[s] = true; }
    });
    return rc;
}

// The same, read back (drawn first if not yet known, as a step would).
int oracle_read_flight(void* p, int s, uint32_t* tc) {
    Handle* h = (Handle*)p;
    DISPATCH(h, {
        O.draw_flights(O.step);
        for (size_t i = 0; i < O.sp[s].size(); ++i) tc[i] = O.sp[s].tc[i];
    });
    return 0;
}

// Host threads of the per-particle loop and the deposit (results do not
// depend on it).  Returns the number of threads OpenMP makes available (1
// when built without it).
int oracle_set_threads(void* p, int n) {
    Handle* h = (Handle*)p;
    DISPATCH(h, O.threads = std::max(1, n));
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// Coulomb collisions (1)-(6): mask bit r-1 enables reaction r, ln_lambda =
// the Coulomb logarithm (a constant of the model).
int oracle_set_coulomb(void* p, uint32_t mask, double ln_lambda) {
    Handle* h = (Handle*)p;
    DISPATCH(h, O.set_coulomb(mask, ln_lambda));
    return 0;
}

int oracle_set_next_id(void* p, int s, uint32_t v) {
    Handle* h = (Handle*)p;
    DISPATCH(h, O.next_id[s] = v);
    return 0;
}

int oracle_step(void* p, uint64_t nsteps) {
    Handle* h = (Handle*)p;
    DISPATCH(h, for (uint64_t k = 0; k < nsteps; ++k) O.do_step());
    return 0;
}

int oracle_set_step(void* p, uint64_t step) {
    Handle* h = (Handle*)p;
    DISPATCH(h, { O.step = step; O.field_valid = false; O.jhist.clear(); });
    return 0;
}

// Conduction-current sums of steps step0 .. step0+n-1 (out[3 i + s]); -1 if
// a step was not recorded since the last load / set_step.
int oracle_currents(void* p, uint64_t step0, uint64_t n, int64_t* out) {
    Handle* h = (Handle*)p; int rc = 0;
    DISPATCH(h, {
        const uint64_t have = O.jhist.size() / NSP;
        if (n > 0 && (O.jhist.empty() || step0 < O.jbase || step0 + n > O.jbase + have)) rc = -1;
        else
            for (uint64_t i = 0; i < n; ++i)
                for (int s = 0; s < NSP; ++s) out[3 * i + s] = O.jhist[(step0 - O.jbase + i) * NSP + s];
    });
    return rc;
}

uint64_t oracle_get_step(void* p) {
    Handle* h = (Handle*)p; uint64_t v = 0;
    DISPATCH(h, v = O.step);
    return v;
}

uint64_t oracle_count(void* p, int s) {
    Handle* h = (Handle*)p; uint64_t v = 0;
    DISPATCH(h, v = O.sp[s].size());
    return v;
}

// Particle state in double (exact for the float mode).
int oracle_read(void* p, int s, double* x, double* vx, double* vy, double* vz, uint32_t* id) {
    Handle* h = (Handle*)p;
    DISPATCH(h, {
        for (size_t i = 0; i < O.sp[s].size(); ++i) {
            x[i] = O.sp[s].x[i]; vx[i] = O.sp[s].vx[i]; vy[i] = O.sp[s].vy[i]; vz[i] = O.sp[s].vz[i];
            id[i] = O.sp[s].id[i];
        }
    });
    return 0;
}

uint64_t oracle_next_id(void* p, int s) {
    Handle* h = (Handle*)p; uint64_t v = 0;
    DISPATCH(h, v = O.next_id[s]);
    return v;
}

// Field of the current step: phi (FP64), E (FP64), and the E copy used by the gather.
int oracle_read_field(void* p, double* phi, double* E, double* Egather) {
    Handle* h = (Handle*)p;
    DISPATCH(h, {
        O.ensure_field();
        for (int j = 0; j < O.Ng; ++j) { phi[j] = O.phi[j]; E[j] = O.Efield[j]; Egather[j] = (double)O.Eg[j]; }
    });
    return 0;
}

// Fixed-point node charges Q[3][Ng] of the current particles and the
// accumulated moments Qacc[3][Ng]; returns the number of accumulated steps.
uint64_t oracle_read_charge(void* p, uint64_t* Q, uint64_t* Qacc) {
    Handle* h = (Handle*)p; uint64_t v = 0;
    DISPATCH(h, {
        O.ensure_field();
        for (int s = 0; s < NSP; ++s)
            for (int j = 0; j < O.Ng; ++j) {
                Q[(size_t)s * O.Ng + j] = O.Q[s][j];
                if (Qacc) Qacc[(size_t)s * O.Ng + j] = O.Qacc[s][j];
            }
        v = O.acc_steps;
    });
    return v;
}

int oracle_reset_moments(void* p) {
    Handle* h = (Handle*)p;
    DISPATCH(h, { for (int s = 0; s < NSP; ++s) std::fill(O.Qacc[s].begin(), O.Qacc[s].end(), 0); O.acc_steps = 0; });
    return 0;
}

// Counters as a flat u64 array; layout = struct Counters.
int oracle_counters(void* p, uint64_t* out, int n) {
    Handle* h = (Handle*)p;
    DISPATCH(h, {
        int m = (int)(sizeof(Counters) / sizeof(uint64_t));
        std::memcpy(out, &O.cnt, sizeof(uint64_t) * (size_t)std::min(n, m));
    });
    return (int)(sizeof(Counters) / sizeof(uint64_t));
}

// Rate table of species s: cumulative rates [NGRID][nproc] (precision R, as
// double), per-process FP64 rates, nu_max and P_max.  Returns nproc.
int oracle_table(void* p, int s, double* cum, double* nu, double* numax, double* pmax) {
    Handle* h = (Handle*)p; int np = 0;
    DISPATCH(h, {
        np = (int)O.procs[s].size();
        for (size_t i = 0; i < (size_t)NGRID * np; ++i) {
            if (cum) cum[i] = (double)O.cum[s][i];
            if (nu) nu[i] = O.nu64[s][i];
        }
        if (numax) *numax = O.numax64[s];
        if (pmax) *pmax = (double)O.Pmax[s];
    });
    return np;
}

int oracle_neutral_table(void* p, double* K) {
    Handle* h = (Handle*)p;
    DISPATCH(h, { for (int i = 0; i < NGRID; ++i) K[i] = (double)O.Ktab[i]; });
    return NGRID;
}

// One particle of species s through push + absorb + MCC at step n with the
// gather field Ef[Ng] (given in double, rounded to R); *tc (in/out) is the
// step of its next collision candidate, drawn afresh at step n as for a
// loaded particle when fresh != 0 (then a candidate with probability P_max).  Returns 1 if the
// particle stays, 0 if it leaves; births (up to 2) are written to
// births[8] = {dst, x, vx, vy, vz, ...} and their number to *nb.  Used for
// sampled checks at sizes where the whole oracle step is too slow.
int oracle_update_particle(void* p, int s, uint64_t n, const double* Ef, double* state, uint32_t id,
                           uint32_t* tc, int fresh, double* births, int* nb) {
    Handle* h = (Handle*)p;
    if (h->f) return update_one<float>(*h->f, s, n, Ef, state, id, tc, fresh, births, nb);
    return update_one<double>(*h->d, s, n, Ef, state, id, tc, fresh, births, nb);
}

// The free-flight gap K (pushes without a candidate) that word w gives for
// species s with the current tables.  Test use.
uint32_t oracle_flight_gap(void* p, int s, uint32_t w) {
    Handle* h = (Handle*)p; uint32_t v = 0;
    DISPATCH(h, v = O.flight_gap(s, w));
    return v;
}

// ---- standalone pieces (pinned directly by tests)
void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    U4 r = philox4x32_10(ctr, key);
    for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

float oracle_ln_f32(float x) { return ln_(x); }

// n samples of the stream helpers (precision 32 or 64): kind 0 = isotropic
// unit vectors (3 per sample), 1 = normal pairs (2 per sample).
void oracle_sample(int kind, int precision, uint32_t seed, uint64_t n, double* out) {
    uint64_t warn = 0;
    for (uint64_t i = 0; i < n; ++i) {
        Stream st((uint32_t)i, seed, 0, 7);
        if (precision == 64) {
            if (kind == 0) { double v[3]; isotropic<double>(st, v, warn); out[3*i] = v[0]; out[3*i+1] = v[1]; out[3*i+2] = v[2]; }
            else { double a, b; normal_pair<double>(st, a, b, warn); out[2*i] = a; out[2*i+1] = b; }
        } else {
            if (kind == 0) { float v[3]; isotropic<float>(st, v, warn); out[3*i] = v[0]; out[3*i+1] = v[1]; out[3*i+2] = v[2]; }
            else { float a, b; normal_pair<float>(st, a, b, warn); out[2*i] = a; out[2*i+1] = b; }
        }
    }
}

void oracle_solve_field(int n_cells, double dx, double weight, double area, double V0,
                        const long long* Rnet, double* phi, double* E) {
    Oracle<double>::solve_field(n_cells, dx, weight, area, V0, Rnet, phi, E);
}

void oracle_solve_field_thomas(int n_cells, double dx, double weight, double area, double V0,
                               const long long* Rnet, double* phi, double* E) {
    Oracle<double>::solve_field_thomas(n_cells, dx, weight, area, V0, Rnet, phi, E);
}

// CIC fixed-point deposit of n float positions onto n_cells+1 nodes.
void oracle_deposit(int n_cells, double L, const float* x, uint64_t n, uint64_t* Q) {
    oracle_config c; std::memset(&c, 0, sizeof(c));
    c.n_cells = n_cells; c.L = L; c.ion_subcycle = 1; c.dt = 1; c.area = 1; c.weight = 1;
    c.m_e = 1; c.m_OM = 1; c.m_OP = 1; c.M_gas = 1; c.T_gas = 1; c.p = 1;
    Oracle<float> O(c);
    std::vector<uint64_t> q(n_cells + 1, 0);
    for (uint64_t i = 0; i < n; ++i) O.deposit_one(q, x[i]);
    for (int j = 0; j <= n_cells; ++j) Q[j] = q[j];
}

// The tabulated rate at an arbitrary energy E [eV], exactly as the collision
// step looks it up (grid_locate + grid_interp in precision R): which = 0..2
// -> cumulative rate column k of species `which`; 3 -> the (17) table sigma_n g;
// 4 -> the (16) table sigma_r g; 5 -> the (22) table sigma_22 g.  Test use
// (pins the lookup off the grid).
double oracle_lookup(void* p, int which, int k, double E) {
    Handle* h = (Handle*)p; double v = 0.0;
    DISPATCH(h, {
        using RR = typename std::remove_reference<decltype(O.Eg[0])>::type;
        int i; RR w; bool above;
        grid_locate<RR>((RR)E, i, w, above);
        if (which >= 0 && which < NSP) {
            const int np = (int)O.procs[which].size();
            if (k >= 0 && k < np) v = (double)O.cum_at(which, k, i, w);
        } else if (which == 3) {
            v = (double)grid_interp<RR>(O.Ktab, 1, 0, i, w);
        } else if (which == 4) {
            v = (double)grid_interp<RR>(O.Ktab_r, 1, 0, i, w);
        } else if (which == 5) {
            v = (double)grid_interp<RR>(O.Ktab_d, 1, 0, i, w);
        }
    });
    return v;
}

double oracle_grid_energy(int i) { return grid_energy(i); }
int oracle_ngrid() { return NGRID; }
int oracle_ncounters() { return (int)(sizeof(Counters) / sizeof(uint64_t)); }

}  // extern "C"
