// o2pic_compact_particles_noalloc: the stable particle compaction of
// o2pic_compact_particles for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a compaction:
// a framework whose caching allocator already holds the free device memory
// (a fresh cudaMalloc fails or fragments it), or a pipeline that keeps
// several streams busy and cannot accept the device-wide synchronization
// that cudaFree implies.  This entry point allocates nothing: its scratch
// (the tile ticket, the live total, an error word and the look-back flag and
// value words) lives in the file-scope array below, sized for at most
// O2PIC_NOALLOC_MAX_PARTICLES particles.  Every GPU that loads the library
// holds this array (about 96 KB) until the process exits.
#include <mutex>

#include "common.cuh"

namespace o2 {
size_t compact_scratch_words(unsigned long long n);
void launch_compact_arrays(const float* x, const float* vx, const float* vy, const float* vz, const uint32_t* id,
                           unsigned long long n, float* ox, float* ovx, float* ovy, float* ovz, uint32_t* oid,
                           unsigned long long* n_out, unsigned long long* words, unsigned long long tiles,
                           unsigned long long epoch, int grid, cudaStream_t s);
}  // namespace o2

using namespace o2;

namespace {

constexpr unsigned long long NOALLOC_MAX_N = O2PIC_NOALLOC_MAX_PARTICLES;
constexpr unsigned long long NOALLOC_TILES = (NOALLOC_MAX_N + TILE - 1) / TILE + 1;
constexpr unsigned long long NOALLOC_WORDS = 3 + 3 * NOALLOC_TILES;

// [ticket, live total, error word, flag[tiles], value[2 * tiles]]
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;

struct DeviceSlot {
    unsigned long long epoch = 0;        // last look-back epoch used on this device
    int sms = 0;
};

std::mutex g_mutex;
DeviceSlot g_slots[MAX_DEVICES];

}  // namespace

extern "C" int o2pic_compact_particles_noalloc(const float* x, const float* vx, const float* vy, const float* vz,
                                               const uint32_t* id, uint64_t n, float* ox, float* ovx, float* ovy,
                                               float* ovz, uint32_t* oid, uint64_t* n_out, void* stream) {
    if (!n_out || (n > 0 && (!x || !vx || !vy || !vz || !id || !ox || !ovx || !ovy || !ovz || !oid)))
        return O2PIC_E_INVALID_ARG;
    if (n > NOALLOC_MAX_N) return O2PIC_E_INVALID_ARG;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return O2PIC_E_CUDA;
    // The host-side name of the array is only a stand-in: its device address
    // on the current device is looked up on every call (cheap), so it stays
    // right even after cudaDeviceReset has reloaded the module.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return O2PIC_E_CUDA;
    unsigned long long* scratch = (unsigned long long*)p;
    unsigned long long epoch;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceSlot& d = g_slots[dev];
        if (d.sms == 0 && cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return O2PIC_E_CUDA;
        // a fresh epoch per call: flags left by earlier calls never match it
        // (after a reset the array is zero again, which no epoch >= 1 matches)
        epoch = ++d.epoch;
        sms = d.sms;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the ticket, the live total and the error word must start at zero
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, sizeof(uint64_t), s);
    if (e == cudaSuccess && n > 0) {
        launch_compact_arrays(x, vx, vy, vz, id, n, ox, ovx, ovy, ovz, oid, (unsigned long long*)n_out, scratch,
                              NOALLOC_TILES, epoch, 4 * sms, s);
        e = cudaGetLastError();
    }
    unsigned long long err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, scratch + 2, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return O2PIC_E_CUDA;
    return (err & ERR_TIMEOUT) ? O2PIC_E_TIMEOUT : O2PIC_OK;
}
