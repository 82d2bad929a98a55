// End-of-step kernel (two blocks): charge commit, cycle moments, Poisson solve
// and E on the nodes; placement of the step's births, removals of (17) and the
// commit of the step; plus the stable compaction of dead slots and small
// utility kernels.
//
// Poisson (Sec. 2): interior nodes satisfy
//     -phi_{j-1} + 2 phi_j - phi_{j+1} = rho_j dx^2 / eps0,
// phi_0 = U sin(2 pi f t) (driven electrode at x = 0), phi_N = 0 (grounded).
// With the net fixed-point charge R_j (2^16 per macro-particle, exact int64)
// and c = e w dx / (A eps0 2^16), the system is solved in closed form by
// exact integer prefix sums (one block-wide scan of the pair S, U):
//     S_m = sum_{k=1..m} R_k,  U_m = sum_{k=1..m} k R_k,
//     T_j = sum_{m<j} S_m = j S_{j-1} - U_{j-1},
//     D_0 = phi_1 - phi_0 = (c T_N - V0) / N,  phi_j = V0 + j D_0 - c T_j,
//     E_j = (c (S_j + S_{j-1}) - 2 D_0) [1/(2 dx)]         (1 <= j <= N-1),
//     E_0 = (-D_0 - c R_0) [1/dx],  E_N = (c S_{N-1} - D_0 + c R_N) [1/dx]
// (wall nodes from Gauss's law over the half cell next to the wall).  This is
// the exact solution of the linear system a Thomas sweep would solve; it
// needs no serial FP64 recurrence (FP64 throughput on this GPU is low), its
// only rounding is in the final FP64 expressions, each evaluated in the order
// written here.  |S| <= 2^47 and |T| <= 2^58 for up to 2^31 particles and 8192
// cells, so int64 holds both exactly.
#include "common.cuh"

namespace o2 {

namespace {

// The end-of-step kernel is two independent blocks of FT threads, each on its
// own SM (twice the memory-level parallelism of one): block 0 commits the
// charge and solves the field, block 1 places the births and commits the step.
// They share nothing; block 0 keeps its own copy of the step counter
// (field_step) for U sin(2 pi f t).
constexpr int FT = 512;
constexpr int GA = FT;                            // threads of the charge block
constexpr int GB = FT;                            // threads of the births block

// Births of one step, placed in the order the method defines (source species
// e then O-, parent order, e before O2+ for an ionization): each warp of a
// particle kernel staged the births of its slot range [u R, ...) with their
// count (their charge already went to Qb there).  The counts are scanned into
// per-warp offsets in shared memory, and every thread of the births block
// then places single births (found by a binary search over the offsets), so
// the work spreads over the block however the births cluster.
// A newborn of step n starts a free flight at its first push after n (step
// n + 1 for electrons, the next ion step for ions), drawn from its own stream
// at step n with tag TAG_FLIGHT + d.
__device__ void place_birth(const Params& P, DevCtrl* C, const unsigned cur[NSP], int d, unsigned long long slot,
                            unsigned long long id64, float4 b, unsigned long long n) {
    const SpeciesBuf& B = P.sp[d];
    if (slot >= B.cap) { atomicOr(&C->error_flags, ERR_CAPACITY); return; }
    // ids are 32-bit: a birth whose id would be 2^32 or more overflows
    // (counted per birth; the particle keeps the low 32 bits)
    if (id64 > 0xFFFFFFFFull) {
        atomicOr(&C->error_flags, ERR_ID);
        atomicAdd(&C->cnt.id_overflow, 1ull);
    }
    const unsigned cb = cur[d];
    const uint32_t id = (uint32_t)id64;
    const unsigned sub = P.sub[d];
    const uint32_t nf = (uint32_t)((n + sub) / sub * sub);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)n, TAG_FLIGHT + (uint32_t)d, 0u, (uint32_t)(n >> 32)),
                                  make_uint2(id, P.seed));
    B.x[cb][slot] = b.x;
    B.vx[cb][slot] = b.y;
    B.vy[cb][slot] = b.z;
    B.vz[cb][slot] = b.w;
    B.id[cb][slot] = id;
    B.tc[cb][slot] = nf + sub * flight_gap(w.x, P.inv_lnq[d], P.kcap[d]);
}

// Exclusive scan over the births block of two 64-bit values per thread, with
// the totals.
__device__ __forceinline__ void groupB_excl_scan_pair(unsigned long long v, unsigned long long w,
                                                      unsigned long long* ws, unsigned long long& ev,
                                                      unsigned long long& ew, unsigned long long& tv,
                                                      unsigned long long& tw) {
    const int tB = threadIdx.x, lane = tB & 31, warp = tB >> 5;
    constexpr int NW = GB / 32;
    unsigned long long x = v, y = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long xo = __shfl_up_sync(0xffffffffu, x, o);
        const unsigned long long yo = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) { x += xo; y += yo; }
    }
    if (lane == 31) { ws[warp] = x; ws[NW + warp] = y; }
    __syncthreads();
    if (warp == 0) {
        unsigned long long a = (lane < NW) ? ws[lane] : 0ull, b = (lane < NW) ? ws[NW + lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long ao = __shfl_up_sync(0xffffffffu, a, o);
            const unsigned long long bo = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ao; b += bo; }
        }
        if (lane < NW) { ws[lane] = a; ws[NW + lane] = b; }
    }
    __syncthreads();
    ev = (warp == 0 ? 0ull : ws[warp - 1]) + x - v;
    ew = (warp == 0 ? 0ull : ws[NW + warp - 1]) + y - w;
    tv = ws[NW - 1];
    tw = ws[2 * NW - 1];
    __syncthreads();
}

// Offsets of the per-warp birth counts: c1, c2 of the electron kernel's nu1
// warps into p1, p2 [0..nu1], c3 of the O- kernel's nu3 warps into p3
// [0..nu3] (nu1 or nu3 may be 0), by one scan over the births block; returns
// the totals (c1 | c2 << 32 and c3).  A thread owns a range of a multiple of 4
// units, read as 16-byte vectors (the count arrays are 256-byte aligned).
__device__ __forceinline__ void unit_range(unsigned nu, unsigned& u0, unsigned& u1) {
    const unsigned tB = threadIdx.x;
    const unsigned per = (((nu + GB - 1) / GB) + 3u) & ~3u;
    u0 = tB * per < nu ? tB * per : nu;
    u1 = (u0 + per < nu) ? u0 + per : nu;
}

__device__ __forceinline__ uint4 count4(const unsigned* c, unsigned u, unsigned nu) {
    if (u + 4 <= nu) return *reinterpret_cast<const uint4*>(c + u);
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (u < nu) r.x = c[u];
    if (u + 1 < nu) r.y = c[u + 1];
    if (u + 2 < nu) r.z = c[u + 2];
    return r;
}

__device__ void unit_offsets(const unsigned* c1, const unsigned* c2, unsigned nu1, const unsigned* c3, unsigned nu3,
                             unsigned* p1, unsigned* p2, unsigned* p3, unsigned long long* ws,
                             unsigned long long& tot12, unsigned long long& tot3) {
    const int tB = threadIdx.x;
    unsigned u0, u1;
    unit_range(nu1 > nu3 ? nu1 : nu3, u0, u1);
    unsigned long long m12 = 0, m3 = 0;
    for (unsigned ub = u0; ub < u1; ub += 8) {
        uint4 a[2], b[2], d[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {       // all loads first
            const unsigned u = ub + 4u * k;
            const bool in = u < u1;
            a[k] = in ? count4(c1, u, nu1) : make_uint4(0u, 0u, 0u, 0u);
            b[k] = in ? count4(c2, u, nu1) : make_uint4(0u, 0u, 0u, 0u);
            d[k] = in ? count4(c3, u, nu3) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const unsigned u = ub + 4u * k;
            const unsigned av[4] = {a[k].x, a[k].y, a[k].z, a[k].w}, bv[4] = {b[k].x, b[k].y, b[k].z, b[k].w},
                           dv[4] = {d[k].x, d[k].y, d[k].z, d[k].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool mine = u + e < u1;   // the next thread's units are its own
                if (mine && u + e < nu1) { p1[u + e] = av[e]; p2[u + e] = bv[e]; }
                if (mine && u + e < nu3) p3[u + e] = dv[e];
                m12 += (unsigned long long)av[e] | ((unsigned long long)bv[e] << 32);
                m3 += dv[e];
            }
        }
    }
    unsigned long long e12, e3;
    groupB_excl_scan_pair(m12, m3, ws, e12, e3, tot12, tot3);
    unsigned r1 = (unsigned)e12, r2 = (unsigned)(e12 >> 32), r3 = (unsigned)e3;
    for (unsigned u = u0; u < u1; ++u) {
        if (u < nu1) { const unsigned x = p1[u], y = p2[u]; p1[u] = r1; p2[u] = r2; r1 += x; r2 += y; }
        if (u < nu3) { const unsigned z = p3[u]; p3[u] = r3; r3 += z; }
    }
    if (tB == 0) { p1[nu1] = (unsigned)tot12; p2[nu1] = (unsigned)(tot12 >> 32); p3[nu3] = (unsigned)tot3; }
    __syncthreads();
}

// Start moving a line into this SM's L1 (the loads that follow hit it).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Prefetch a births-block thread's share [u0, u1) of the per-warp counts
// (the lines of its first and last unit: a share spans at most two lines
// while it holds at most 32 units).
__device__ __forceinline__ void prefetch_units(const unsigned* c1, const unsigned* c2, unsigned nu1, const unsigned* c3,
                                               unsigned nu3) {
    unsigned u0, u1;
    unit_range(nu1 > nu3 ? nu1 : nu3, u0, u1);
    if (u0 >= u1) return;
    const unsigned ends[2] = {u0, u1 - 1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned u = ends[k];
        if (u < nu1) { prefetch_l1(c1 + u); prefetch_l1(c2 + u); }
        if (u < nu3) prefetch_l1(c3 + u);
    }
}

// The warp that staged birth number b (largest u with p[u] <= b).
__device__ __forceinline__ unsigned find_unit(const unsigned* p, unsigned nu, unsigned b) {
    unsigned lo = 0, hi = nu;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (p[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

struct CtrlSnap {
    unsigned long long step, epoch, acc_steps, slots[NSP], live[NSP], removed[NSP];
    unsigned long long next_id[NSP];
    unsigned cur[NSP], removals, births22;
};

// Over the charge block: the inclusive scan S_j of R_j held in a[0..n)
// (a[0] = 0; in place), and U_j = sum_{k<=j} k R_k straight to global U[j]
// (its only readers are the potential and D0, which gets U_{n-2} in *u_last).
// Blocked: thread t owns [t*per, (t+1)*per); the two scans share their
// warp shuffles and barriers.
__device__ __forceinline__ void groupA_scan_SU(long long* a, int n, long long* ws, long long* U, long long* u_last) {
    const int t = threadIdx.x;
    const int per = (n + GA - 1) / GA;
    const int j0 = t * per;
    long long ra = 0, rb = 0;
    for (int i = 0; i < per; ++i) {
        const int j = j0 + i;
        if (j < n) { const long long r = a[j]; ra += r; a[j] = ra; rb += (long long)j * r; }
    }
    const int lane = t & 31, warp = t >> 5;
    long long xa = ra, xb = rb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long ya = __shfl_up_sync(0xffffffffu, xa, o);
        const long long yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) { xa += ya; xb += yb; }
    }
    if (lane == 31) { ws[warp] = xa; ws[32 + warp] = xb; }
    __syncthreads();
    if (warp == 0) {
        long long va = (lane < GA / 32) ? ws[lane] : 0, vb = (lane < GA / 32) ? ws[32 + lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long ya = __shfl_up_sync(0xffffffffu, va, o);
            const long long yb = __shfl_up_sync(0xffffffffu, vb, o);
            if (lane >= o) { va += ya; vb += yb; }
        }
        if (lane < GA / 32) { ws[lane] = va; ws[32 + lane] = vb; }
    }
    __syncthreads();
    const long long offa = (warp == 0 ? 0 : ws[warp - 1]) + (xa - ra);
    const long long offb = (warp == 0 ? 0 : ws[32 + warp - 1]) + (xb - rb);
    long long prev = 0, ub = 0;
    for (int i = 0; i < per; ++i) {
        const int j = j0 + i;
        if (j < n) {
            const long long sl = a[j];          // thread-local inclusive S
            ub += (long long)j * (sl - prev);
            prev = sl;
            a[j] = sl + offa;
            U[j] = ub + offb;
            if (j == n - 2) *u_last = ub + offb;
        }
    }
    __syncthreads();
}

// mode 0: end of a step (pushed_mask = species pushed this step);
// mode 1: after a load (all species freshly deposited into Qf).
// Dynamic shared memory: S as int64 [Ng] (charge group), then three u32
// [max warps + 1] (births group).
__device__ __forceinline__ void field_body(const Params& P, int mode, int pushed_mask, int role) {
    extern __shared__ long long fsm[];
    __shared__ long long wsA[64];
    __shared__ unsigned long long wsB[2 * (GB / 32)];
    __shared__ CtrlSnap cs;
    __shared__ long long sh_R0, sh_RN, sh_UN1;
    __shared__ double sh_V0, sh_D0;
    __shared__ unsigned long long sh_fstep;
    DevCtrl* C = P.ctrl;
    const int N = P.Nc, Ng = P.Ng;
    const int t = threadIdx.x;

    if (role == 0) {
        // ================= charge commit, cycle moments, field solve
        long long* Ss = fsm;          // S_j = sum_{k=1..j} R_k   (T_j = j S_{j-1} - U_{j-1})
        if (t == 0) {
            // U sin(2 pi f t) at t^{n+1} (end of step) or t^n (after a load),
            // evaluated on the host in FP64 and staged in a ring indexed by
            // the step
            const unsigned long long fstep = C->field_step;
            sh_fstep = fstep;
            sh_V0 = P.vring[(mode == 0 ? fstep + 1 : fstep) & P.vring_mask];
        }
        // Q = (this step's deposit Qf, or the kept Q of a species not pushed)
        // + the births' deposit Qb, and the cycle moments Qacc += Q; two
        // nodes per thread with all their loads issued before any store
        for (int j0 = t; j0 < Ng; j0 += 2 * GA) {
            unsigned long long q[2][NSP], qa[2][NSP];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h * GA;
#pragma unroll
                for (int s = 0; s < NSP; ++s) {
                    q[h][s] = 0ull;
                    qa[h][s] = 0ull;
                    if (j < Ng) {
                        if (mode == 0) qa[h][s] = P.Qacc[s][j];
                        const bool fresh = (mode == 1) || ((pushed_mask >> s) & 1);
                        unsigned long long v = P.Qb[s][j];
                        if (fresh) {
#pragma unroll
                            for (int k = 0; k < QCOPIES; ++k) v += P.Qf[s][(size_t)k * Ng + j];
                        } else {
                            v += P.Q[s][j];
                        }
                        q[h][s] = v;
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h * GA;
                if (j >= Ng) continue;
                long long net = 0;
#pragma unroll
                for (int s = 0; s < NSP; ++s) {
                    P.Q[s][j] = q[h][s];
                    if (mode == 0) P.Qacc[s][j] = qa[h][s] + q[h][s];
                    P.Qf[s][j] = 0ull;
                    if ((mode == 1) || ((pushed_mask >> s) & 1)) {   // only pushes fill copies 1..
#pragma unroll
                        for (int k = 1; k < QCOPIES; ++k) P.Qf[s][(size_t)k * Ng + j] = 0ull;
                    }
                    P.Qb[s][j] = 0ull;
                    net += (s == SP_OP) ? (long long)q[h][s] : -(long long)q[h][s];
                }
                Ss[j] = (j >= 1) ? net : 0;                    // scanned below
                if (j == 0) sh_R0 = net;
                if (j == N) sh_RN = net;
            }
        }
        __syncthreads();
        groupA_scan_SU(Ss, Ng, wsA, P.fU, &sh_UN1);
        const double c = P.c_field;
        // D0 once per block: FP64 throughput on this GPU is low
        if (t == 0) {
            const long long TN = (long long)N * Ss[N - 1] - sh_UN1;
            // a power-of-two N divides exactly by its reciprocal (same IEEE
            // result as the division, which is slow in FP64 here)
            const double num = c * (double)TN - sh_V0;
            const double D0 = (P.inv_Nc64 != 0.0) ? num * P.inv_Nc64 : num / (double)N;
            sh_D0 = D0;
            P.fVD[0] = sh_V0;
            P.fVD[1] = D0;
            if (mode == 0) C->field_step = sh_fstep + 1;   // only this block reads it
        }
        __syncthreads();
        // E on the nodes (what the next push gathers).  The potential needs as
        // much FP64 work again and only diagnostics read it: S, U, V0 and D0
        // are kept so that k_phi evaluates it with the same expressions.
        const double D0 = sh_D0, D2 = 2.0 * sh_D0;   // 2 D0 is exact
        const long long R0 = sh_R0, RN = sh_RN;
        for (int j = t; j < Ng; j += GA) {
            double E;
            if (j == 0) E = (-D0 - c * (double)R0) * P.inv_dx64;
            else if (j == N) E = (c * (double)Ss[N - 1] - D0 + c * (double)RN) * P.inv_dx64;
            else E = (c * (double)(Ss[j] + Ss[j - 1]) - D2) * P.inv_2dx64;
            P.Ef[j] = (float)E;
            P.fS[j] = Ss[j];
        }
        return;
    }

    // ===================== births, (17) removals and the commit of the step
    const int tB = t;
    unsigned* p1 = reinterpret_cast<unsigned*>(fsm + Ng);
    unsigned* p2 = p1 + (P.max_push_warps + 1);
    unsigned* p3 = p2 + (P.max_push_warps + 1);
    const bool births_e = mode == 0 && P.births_possible[SP_E];
    const bool births_om = mode == 0 && ((pushed_mask >> SP_OM) & 1) && P.births_possible[SP_OM];
    if (tB < NSP) {
        cs.slots[tB] = C->slots[tB]; cs.live[tB] = C->live[tB]; cs.removed[tB] = C->removed[tB];
        cs.next_id[tB] = C->next_id[tB]; cs.cur[tB] = C->cur[tB];
    } else if (tB == 32) {
        cs.step = C->step;
        cs.epoch = C->epoch;
        cs.acc_steps = C->acc_steps;
        cs.removals = C->removals;
        cs.births22 = C->births22;
    }
    prefetch_units(P.wcount[B_E_FROM_E], P.wcount[B_OM_FROM_E], births_e ? P.push_warps[SP_E] : 0u,
                   P.wcount[B_E_FROM_OM], births_om ? P.push_warps[SP_OM] : 0u);
    __syncthreads();

    // births of the step: n1 ionizations (e + O2+) and n2 attachments (O-)
    // staged by the electron kernel, n3 detachment electrons staged by the O-
    // kernel (ion steps), placed after the electrons' own, then n4 electrons
    // of (22) staged in order by its apply kernel (ion steps)
    unsigned long long btot[NB];
    for (int k = 0; k < NB; ++k) btot[k] = 0;
    const unsigned n4 = (mode == 0) ? cs.births22 : 0u;
    if (births_e || births_om || n4) {
        const unsigned ns1 = (unsigned)(cs.slots[SP_E] < P.sp[SP_E].cap ? cs.slots[SP_E] : P.sp[SP_E].cap);
        const unsigned ns3 = (unsigned)(cs.slots[SP_OM] < P.sp[SP_OM].cap ? cs.slots[SP_OM] : P.sp[SP_OM].cap);
        const unsigned nu1 = births_e ? P.push_warps[SP_E] : 0u, nu3 = births_om ? P.push_warps[SP_OM] : 0u;
        const unsigned R1 = warp_range_len(ns1, nu1 ? nu1 : 1u), R3 = warp_range_len(ns3, nu3 ? nu3 : 1u);
        unsigned long long t12, t3;
        unit_offsets(P.wcount[B_E_FROM_E], P.wcount[B_OM_FROM_E], nu1, P.wcount[B_E_FROM_OM], nu3, p1, p2, p3, wsB,
                     t12, t3);
        const unsigned n1 = (unsigned)t12, n2 = (unsigned)(t12 >> 32), n3 = (unsigned)t3;
        const unsigned ntot = n1 + n2 + n3 + n4;
        // one birth per thread and pass: which list, its rank there, the warp
        // that staged it (binary search over that list's offsets) and its
        // staging slot; all loads of the birth before its stores
        for (unsigned b = tB; b < ntot; b += GB) {
            if (b >= n1 + n2 + n3) {   // (22): staged in place order
                const unsigned r = b - n1 - n2 - n3;
                place_birth(P, C, cs.cur, SP_E, cs.slots[SP_E] + n1 + n3 + r,
                            (unsigned long long)cs.next_id[SP_E] + n1 + n3 + r, P.stage22[r], cs.step);
                continue;
            }
            const int kind = b < n1 ? 0 : (b < n1 + n2 ? 1 : 2);
            const unsigned r = kind == 0 ? b : (kind == 1 ? b - n1 : b - n1 - n2);
            const unsigned* p = kind == 0 ? p1 : (kind == 1 ? p2 : p3);
            const unsigned nu = kind == 2 ? nu3 : nu1, R = kind == 2 ? R3 : R1, ns = kind == 2 ? ns3 : ns1;
            const unsigned u = find_unit(p, nu, r);
            const unsigned long long sb = ((unsigned long long)u * R < ns ? (unsigned long long)u * R : ns) + (r - p[u]);
            if (kind == 0) {
                const float4 be = P.stage[B_E_FROM_E][sb], bo = P.stage[B_OP_FROM_E][sb];
                place_birth(P, C, cs.cur, SP_E, cs.slots[SP_E] + r, (unsigned long long)cs.next_id[SP_E] + r, be,
                            cs.step);
                place_birth(P, C, cs.cur, SP_OP, cs.slots[SP_OP] + r, (unsigned long long)cs.next_id[SP_OP] + r, bo,
                            cs.step);
            } else if (kind == 1) {
                place_birth(P, C, cs.cur, SP_OM, cs.slots[SP_OM] + r, (unsigned long long)cs.next_id[SP_OM] + r,
                            P.stage[B_OM_FROM_E][sb], cs.step);
            } else {
                place_birth(P, C, cs.cur, SP_E, cs.slots[SP_E] + n1 + r, (unsigned long long)cs.next_id[SP_E] + n1 + r,
                            P.stage[B_E_FROM_OM][sb], cs.step);
            }
        }
        btot[B_E_FROM_E] = n1;
        btot[B_OP_FROM_E] = n1;
        btot[B_OM_FROM_E] = n2;
        btot[B_E_FROM_OM] = n3 + n4;
    }

    if (mode == 0) {
        // (17) removals: mark both ions of every reacted pair dead
        const unsigned nrem = (cs.removals < P.max_removals) ? cs.removals : P.max_removals;
        for (unsigned r = tB; r < nrem; r += GB) {
            P.sp[SP_OM].x[cs.cur[SP_OM]][P.removal[2 * r]] = dead_marker();
            P.sp[SP_OP].x[cs.cur[SP_OP]][P.removal[2 * r + 1]] = dead_marker();
        }
        // commit of the step: one thread per species, then the step counters
        if (tB < NSP) {
            const int s = tB;
            const unsigned long long bs = (s == SP_E) ? btot[B_E_FROM_E] + btot[B_E_FROM_OM]
                                                      : (s == SP_OP ? btot[B_OP_FROM_E] : btot[B_OM_FROM_E]);
            const unsigned long long rem = cs.removed[s] + ((s != SP_E) ? (unsigned long long)nrem : 0ull);
            unsigned long long ns = cs.slots[s] + bs;
            unsigned long long nl = cs.live[s] + bs - rem;
            if (ns > P.sp[s].cap) {   // births beyond the capacity were dropped
                atomicOr(&C->error_flags, ERR_CAPACITY);
                nl -= (ns - P.sp[s].cap) < nl ? (ns - P.sp[s].cap) : nl;
                ns = P.sp[s].cap;
            }
            C->slots[s] = ns;
            C->live[s] = nl;
            C->next_id[s] = cs.next_id[s] + bs;
            C->removed[s] = 0ull;
            if (bs) atomicAdd(&C->cnt.born[s], bs);
        } else if (tB == 32) {
            if (nrem) atomicAdd(&C->cnt.neutralized, (unsigned long long)nrem);
            // this block is the only writer of the step state: plain stores
            C->removals = 0u;
            C->rremovals = 0u;
            C->dremovals = 0u;
            C->births22 = 0u;
            C->acc_steps = cs.acc_steps + 1;
            C->step = cs.step + 1;
            C->epoch = cs.epoch + 1;
        } else if (tB >= 64 && tB < 64 + NKK + NSP) {
            C->ticket[tB - 64] = 0u;
        }
    }
    // per-cell ion totals of (17): zero for the next ion step
    for (int k = tB; k < 2 * N; k += GB) { P.ptot[k] = 0u; P.rtot[k] = 0u; P.dtot[k] = 0u; }
    // conduction-current sums: after a load the ring restarts; at the end of
    // step n the ions' entries of a step without an ion push repeat those of
    // step n-1, and the slot of step n+1 is cleared for its pushes
    if (mode != 0) {
        for (int k = tB; k < JRING * NSP; k += GB) P.jring[k] = 0ull;
        if (tB < NKK + NSP) C->ticket[tB] = 0u;
    } else if (tB >= 96 && tB < 96 + NSP) {
        const int sp = tB - 96;
        const unsigned long long n = cs.step;
        if (sp != SP_E && !((pushed_mask >> sp) & 1))
            P.jring[(n & (JRING - 1)) * NSP + sp] = P.jring[((n - 1) & (JRING - 1)) * NSP + sp];
        P.jring[((n + 1) & (JRING - 1)) * NSP + sp] = 0ull;
    }
}

// Stable compaction of the live slots of one species into the other buffer
// (mode 0, when more than a fraction of the slots is dead), or a stable copy
// of the live particles into caller buffers (mode 1).  Tiles of TILE slots in
// increasing order, decoupled look-back on the live counts.
template <int S>
__device__ __forceinline__ void compact_body(const Params& P, int mode, unsigned long long epoch_arg,
                                             unsigned* ticket_arg, unsigned long long* flag_arg,
                                             unsigned long long* val_arg, float* ox, float* ovx, float* ovy,
                                             float* ovz, uint32_t* oid, uint32_t* otc, unsigned long long ocap,
                                             unsigned long long* out_count) {
    __shared__ unsigned ws[32];
    __shared__ unsigned sh_tile;
    __shared__ unsigned long long sh_excl;
    __shared__ int sh_ok;
    DevCtrl* C = P.ctrl;
    const unsigned long long nslots = C->slots[S];
    const unsigned long long live = C->live[S];
    if (mode == 0) {
        const unsigned long long dead = nslots - live;
        const bool many_dead = (double)dead > (double)P.compact_dead_frac * (double)nslots;
        const bool near_full = dead > 0 && 4 * nslots > 3 * P.sp[S].cap;
        if (!many_dead && !near_full) return;
    }
    const unsigned cb = C->cur[S];
    const float* X = P.sp[S].x[cb];
    const float* VX = P.sp[S].vx[cb];
    const float* VY = P.sp[S].vy[cb];
    const float* VZ = P.sp[S].vz[cb];
    const uint32_t* ID = P.sp[S].id[cb];
    const uint32_t* TCS = P.sp[S].tc[cb];
    float *DX, *DVX, *DVY, *DVZ; uint32_t *DID, *DTC;
    unsigned long long dcap;
    unsigned* ticket; unsigned long long *flag, *val, epoch;
    if (mode == 0) {
        DX = P.sp[S].x[cb ^ 1u]; DVX = P.sp[S].vx[cb ^ 1u]; DVY = P.sp[S].vy[cb ^ 1u]; DVZ = P.sp[S].vz[cb ^ 1u];
        DID = P.sp[S].id[cb ^ 1u]; DTC = P.sp[S].tc[cb ^ 1u]; dcap = P.sp[S].cap;
        ticket = &C->ticket[NKK + S];
        flag = P.lb_flag[KK_COMPACT]; val = P.lb_val[KK_COMPACT];
        epoch = (C->epoch << 2) | (unsigned long long)S;
    } else {
        DX = ox; DVX = ovx; DVY = ovy; DVZ = ovz; DID = oid; DTC = otc; dcap = ocap;
        ticket = ticket_arg; flag = flag_arg; val = val_arg; epoch = epoch_arg;
    }
    const unsigned ntiles = (unsigned)ceil_div(nslots, TILE);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh_tile = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned tile = sh_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        const unsigned long long base = (unsigned long long)tile * TILE;
        const unsigned long long end = (base + TILE < nslots) ? base + TILE : nslots;
        // pass 1: live count of the tile
        unsigned cnt = 0;
        for (int c = 0; c < CHUNKS_PER_TILE; ++c) {
            const unsigned long long i0 = base + (unsigned long long)c * CHUNK + 4ull * tid;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i0 + k < end && !is_dead(X[i0 + k])) ++cnt;
        }
        unsigned tile_total;
        (void)block_excl_scan<BLOCK>(cnt, ws, &tile_total);
        if (tid == 0) {
            bool ok;
            sh_excl = lookback(flag, val, tile, pack2(tile_total, 0u), epoch, &C->error_flags, &ok);
            sh_ok = ok ? 1 : 0;
            if (ok && tile == ntiles - 1) {
                const unsigned long long total = (unsigned)sh_excl + (unsigned long long)tile_total;
                if (mode == 0) {
                    C->slots[S] = total;
                    C->live[S] = total;
                    C->cur[S] = cb ^ 1u;
                } else {
                    *out_count = total;
                }
            }
        }
        __syncthreads();
        if (sh_ok) {
            // pass 2: destinations in slot order, chunk by chunk in (thread, k) order
            unsigned long long run = (unsigned)sh_excl;
            for (int c = 0; c < CHUNKS_PER_TILE; ++c) {
                const unsigned long long i0 = base + (unsigned long long)c * CHUNK + 4ull * tid;
                unsigned m = 0;
                bool lv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) { lv[k] = (i0 + k < end) && !is_dead(X[i0 + k]); m += lv[k] ? 1u : 0u; }
                unsigned ctot;
                const unsigned off = block_excl_scan<BLOCK>(m, ws, &ctot);
                unsigned long long d = run + off;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!lv[k]) continue;
                    if (d < dcap) {
                        // a gather (mode 1) may ask for the flights only
                        if (DX) {
                            DX[d] = X[i0 + k]; DVX[d] = VX[i0 + k]; DVY[d] = VY[i0 + k]; DVZ[d] = VZ[i0 + k];
                            DID[d] = ID[i0 + k];
                        }
                        if (DTC) DTC[d] = TCS[i0 + k];
                    }
                    ++d;
                }
                run += ctot;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(FT) k_field(Params P, int mode, int pushed_mask) {
    pdl_wait();
    pdl_trigger();   // two blocks on two SMs: the next step's push may take the others
    field_body(P, mode, pushed_mask, (int)blockIdx.x);
}

// batched: blocks 2d and 2d + 1 are the end-of-step kernel of discharge d
__global__ void __launch_bounds__(FT) k_field_b(const Params* __restrict__ all, int mode, int pushed_mask) {
    __shared__ Params sP;
    pdl_wait();
    pdl_trigger();
    load_params(sP, all + (blockIdx.x >> 1));
    field_body(sP, mode, pushed_mask, (int)(blockIdx.x & 1u));
}

template <int S>
__global__ void __launch_bounds__(BLOCK) k_compact(Params P, int mode, unsigned long long epoch_arg, unsigned* ticket_arg,
                                                   unsigned long long* flag_arg, unsigned long long* val_arg, float* ox,
                                                   float* ovx, float* ovy, float* ovz, uint32_t* oid, uint32_t* otc,
                                                   unsigned long long ocap, unsigned long long* out_count) {
    pdl_wait();
    compact_body<S>(P, mode, epoch_arg, ticket_arg, flag_arg, val_arg, ox, ovx, ovy, ovz, oid, otc, ocap, out_count);
}

// batched compaction check (mode 0): the blocks of map[b].x claim that
// discharge's tiles by its own ticket
template <int S>
__global__ void __launch_bounds__(BLOCK) k_compact_b(const Params* __restrict__ all, const uint4* __restrict__ map) {
    __shared__ Params sP;
    pdl_wait();
    load_params(sP, all + map[blockIdx.x].x);
    compact_body<S>(sP, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr);
}

// Validation of freshly loaded particles (x in [0, L), finite velocities)
// and the largest id (+1) for the species' next id.
template <int S>
__global__ void k_load_check(Params P, unsigned long long n) {
    DevCtrl* C = P.ctrl;
    const unsigned cb = C->cur[S];
    const float* X = P.sp[S].x[cb];
    const float* VX = P.sp[S].vx[cb];
    const float* VY = P.sp[S].vy[cb];
    const float* VZ = P.sp[S].vz[cb];
    const uint32_t* ID = P.sp[S].id[cb];
    unsigned long long mx = 0;
    bool bad = false;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float x = X[i];
        if (!(x >= 0.0f && x < P.Lf) || !isfinite(VX[i]) || !isfinite(VY[i]) || !isfinite(VZ[i])) bad = true;
        const unsigned long long v = (unsigned long long)ID[i] + 1ull;
        mx = v > mx ? v : mx;
    }
    if (bad) atomicOr(&C->error_flags, ERR_NONFINITE);
    atomicMax(&C->next_id[S], mx);
}

__global__ void k_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 r = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}

__global__ void k_ln(const float* x, float* out, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        out[i] = ln_series(x[i]);
}

}  // namespace

size_t field_smem_bytes(const Params& P) {
    return sizeof(long long) * (size_t)P.Ng + 3 * sizeof(unsigned) * ((size_t)P.max_push_warps + 1);
}

// The potential of the last field solve: phi_0 = V0, phi_N = 0,
// phi_j = V0 + j D0 - c T_j with T_j = j S_{j-1} - U_{j-1} (FP64, the
// expressions of the closed-form solve).
__global__ void k_phi(Params P) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.Nc;
    if (j > N) return;
    const double V0 = P.fVD[0], D0 = P.fVD[1], c = P.c_field;
    const long long Tj = (j >= 1) ? (long long)j * P.fS[j - 1] - P.fU[j - 1] : 0;
    P.phi[j] = (j == 0) ? V0 : (j == N ? 0.0 : V0 + (double)j * D0 - c * (double)Tj);
}

void launch_phi(const Params& P, cudaStream_t s) {
    k_phi<<<(P.Ng + 255) / 256, 256, 0, s>>>(P);
}

void launch_field_batched(const Params* all, int n, size_t smem, int mode, int pushed_mask, cudaStream_t s) {
    launch_pdl(k_field_b, 2 * n, FT, smem, s, all, mode, pushed_mask);
}

void launch_compact_batched(int species, const Params* all, const uint4* map, int nblocks, cudaStream_t s) {
    auto k = species == SP_E ? k_compact_b<SP_E> : (species == SP_OM ? k_compact_b<SP_OM> : k_compact_b<SP_OP>);
    launch_pdl(k, nblocks, BLOCK, 0, s, all, map);
}

void launch_field(const Params& P, int mode, int pushed_mask, cudaStream_t s) {
    launch_pdl(k_field, 2, FT, field_smem_bytes(P), s, P, mode, pushed_mask);
}

cudaError_t configure_field_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_field_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

void launch_compact(int species, const Params& P, int grid, cudaStream_t s) {
    auto k = species == SP_E ? k_compact<SP_E> : (species == SP_OM ? k_compact<SP_OM> : k_compact<SP_OP>);
    launch_pdl(k, grid, BLOCK, 0, s, P, 0, 0ull, (unsigned*)nullptr, (unsigned long long*)nullptr,
               (unsigned long long*)nullptr, (float*)nullptr, (float*)nullptr, (float*)nullptr, (float*)nullptr,
               (uint32_t*)nullptr, (uint32_t*)nullptr, 0ull, (unsigned long long*)nullptr);
}

void launch_gather(int species, const Params& P, int grid, unsigned long long epoch, unsigned* ticket,
                   unsigned long long* flag, unsigned long long* val, float* x, float* vx, float* vy, float* vz,
                   uint32_t* id, uint32_t* tc, unsigned long long cap, unsigned long long* out_count, cudaStream_t s) {
    if (species == SP_E)
        k_compact<SP_E><<<grid, BLOCK, 0, s>>>(P, 1, epoch, ticket, flag, val, x, vx, vy, vz, id, tc, cap, out_count);
    else if (species == SP_OM)
        k_compact<SP_OM><<<grid, BLOCK, 0, s>>>(P, 1, epoch, ticket, flag, val, x, vx, vy, vz, id, tc, cap, out_count);
    else
        k_compact<SP_OP><<<grid, BLOCK, 0, s>>>(P, 1, epoch, ticket, flag, val, x, vx, vy, vz, id, tc, cap, out_count);
}

void launch_load_check(int species, const Params& P, unsigned long long n, cudaStream_t s) {
    const int grid = (int)(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096);
    if (species == SP_E) k_load_check<SP_E><<<grid, 256, 0, s>>>(P, n);
    else if (species == SP_OM) k_load_check<SP_OM><<<grid, 256, 0, s>>>(P, n);
    else k_load_check<SP_OP><<<grid, 256, 0, s>>>(P, n);
}

void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, unsigned long long n, cudaStream_t s) {
    const int grid = (int)(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096);
    k_philox<<<grid, 256, 0, s>>>(ctr, key, out, n);
}

void launch_ln(const float* x, float* out, unsigned long long n, cudaStream_t s) {
    const int grid = (int)(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096);
    k_ln<<<grid, 256, 0, s>>>(x, out, n);
}

}  // namespace o2
