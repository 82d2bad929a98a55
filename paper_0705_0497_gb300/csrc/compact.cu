// Stable compaction of a caller's particle arrays (the removal half of the
// method's births/removal step): particles whose x is NaN (the library's
// marker of a removed particle) are dropped, the others are written in their
// original order to the output arrays.  One pass over tiles of TILE
// particles claimed in increasing order; each tile's live count is combined
// with the earlier tiles' by a decoupled look-back.  The look-back state and
// the tile ticket are the kernel's scratch memory.
#include "common.cuh"

namespace o2 {

namespace {

__global__ void __launch_bounds__(BLOCK) k_compact_arrays(const float* __restrict__ X, const float* __restrict__ VX,
                                                          const float* __restrict__ VY, const float* __restrict__ VZ,
                                                          const uint32_t* __restrict__ ID, unsigned long long n,
                                                          float* OX, float* OVX, float* OVY, float* OVZ, uint32_t* OID,
                                                          unsigned long long* n_out, unsigned long long* ticket,
                                                          unsigned long long* count, unsigned long long* flag,
                                                          unsigned long long* val, unsigned long long epoch,
                                                          unsigned long long* err) {
    __shared__ unsigned ws[32];
    __shared__ unsigned sh_tile;
    __shared__ unsigned long long sh_excl;
    __shared__ int sh_ok;
    const unsigned ntiles = (unsigned)ceil_div(n, TILE);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh_tile = (unsigned)atomicAdd(ticket, 1ull);
        __syncthreads();
        const unsigned tile = sh_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        const unsigned long long base = (unsigned long long)tile * TILE;
        const unsigned long long end = (base + TILE < n) ? base + TILE : n;
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
            sh_excl = lookback(flag, val, tile, pack2(tile_total, 0u), epoch, err, &ok);
            sh_ok = ok ? 1 : 0;
            if (ok && tile == ntiles - 1) {
                const unsigned long long total = (unsigned)sh_excl + (unsigned long long)tile_total;
                *count = total;
                *n_out = total;
            }
        }
        __syncthreads();
        if (sh_ok) {
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
                    OX[d] = X[i0 + k]; OVX[d] = VX[i0 + k]; OVY[d] = VY[i0 + k]; OVZ[d] = VZ[i0 + k];
                    OID[d] = ID[i0 + k];
                    ++d;
                }
                run += ctot;
            }
        }
        __syncthreads();
    }
}

// One thread waits, as tile 1 of a look-back, for tile 0, whose flag nothing
// ever sets (epoch 1 against the zeroed flag): the bounded wait must give up,
// set the timeout bit and return.  words = [err, flag[2], val[4]].
__global__ void k_lookback_probe(unsigned long long* words) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool ok;
    (void)lookback(words + 1, words + 3, 1u, pack2(1u, 0u), 1ull, words, &ok);
}

}  // namespace

size_t compact_scratch_words(unsigned long long n) {
    const unsigned long long tiles = ceil_div(n, TILE) + 1;
    return 3 + 3 * tiles;   // ticket, count, error word, flags, values
}

// Scratch laid out in `words` (u64): [ticket, count, err, flag[tiles], val[2 tiles]].
void launch_compact_arrays(const float* x, const float* vx, const float* vy, const float* vz, const uint32_t* id,
                           unsigned long long n, float* ox, float* ovx, float* ovy, float* ovz, uint32_t* oid,
                           unsigned long long* n_out, unsigned long long* words, unsigned long long tiles,
                           unsigned long long epoch, int grid, cudaStream_t s) {
    k_compact_arrays<<<grid, BLOCK, 0, s>>>(x, vx, vy, vz, id, n, ox, ovx, ovy, ovz, oid, n_out, &words[0], &words[1],
                                            &words[3], &words[3 + tiles], epoch, &words[2]);
}

}  // namespace o2

using namespace o2;

extern "C" int o2pic_check_bounded_wait(double* seconds, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* w = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&w, 7 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, 7 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_lookback_probe<<<1, 32, 0, s>>>(w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    unsigned long long err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, w, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (seconds) *seconds = 1e-3 * ms;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (w) cudaFree(w);
    if (e != cudaSuccess) return O2PIC_E_CUDA;
    return (err & ERR_TIMEOUT) ? O2PIC_E_TIMEOUT : O2PIC_OK;
}

extern "C" int o2pic_compact_particles(const float* x, const float* vx, const float* vy, const float* vz,
                                       const uint32_t* id, uint64_t n, float* ox, float* ovx, float* ovy, float* ovz,
                                       uint32_t* oid, uint64_t* n_out, void* stream) {
    if (!n_out || (n > 0 && (!x || !vx || !vy || !vz || !id || !ox || !ovx || !ovy || !ovz || !oid)))
        return O2PIC_E_INVALID_ARG;
    if (n > (1ull << 31)) return O2PIC_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long tiles = ceil_div(n, TILE) + 1;
    const size_t words = compact_scratch_words(n);
    unsigned long long* scratch = nullptr;
    cudaError_t e = cudaMalloc((void**)&scratch, sizeof(unsigned long long) * words);
    if (e != cudaSuccess) return O2PIC_E_CUDA;
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, sizeof(uint64_t), s);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && n > 0) {
        launch_compact_arrays(x, vx, vy, vz, id, n, ox, ovx, ovy, ovz, oid, (unsigned long long*)n_out, scratch, tiles,
                              1ull, 4 * sms, s);
        e = cudaGetLastError();
    }
    unsigned long long err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &scratch[2], sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) return O2PIC_E_CUDA;
    return (err & ERR_TIMEOUT) ? O2PIC_E_TIMEOUT : O2PIC_OK;
}
