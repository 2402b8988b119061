// bisp_cell_order_noalloc: the stable cell ordering of bisp_cell_order for callers that
// cannot allocate device memory (for example code running inside a memory pool or a
// framework that forbids cudaMalloc during a step, or callers without allocation
// rights on the device).  Its scratch lives in one file-scope device array of a fixed
// size, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <exception>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bisp.h"
#include "common.cuh"
#include "internal.h"

namespace {

// Largest catalogue the call accepts, and the scratch it needs for it (bytes):
// keys + indices (8 B), offsets (16 B), radix-sort ping-pong (8 B) per particle, plus the
// sort histograms, scan sums, FP64 partials, the error counter and a y_l^m table.
constexpr int64_t kMaxParticles = BISP_NOALLOC_MAX_PARTICLES;
constexpr size_t kScratchBytes = (size_t)kMaxParticles * 32 + ((size_t)4 << 20);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;  // device address of the array, per device ordinal

// device address of the scratch array on the current device (set up once per device)
void* scratch_address(int* status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *status = BISP_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *status = BISP_ECUDA;
      return nullptr;
    }
    g_addr[dev] = p;
  }
  *status = BISP_OK;
  return g_addr[dev];
}

}  // namespace

extern "C" bisp_status bisp_cell_order_noalloc(int nmesh, double box_len, int mas, const float* xyz, int64_t n,
                                                uint32_t* keys_out, uint32_t* order_out, void* stream) {
  using namespace bisp;
  try {
    if (nmesh < 16 || nmesh > BISP_NMAX || (nmesh & (nmesh - 1))) throw Error{BISP_EINVAL, "nmesh"};
    if (!(box_len > 0)) throw Error{BISP_EINVAL, "box_len"};
    if (mas < 1 || mas > 3) throw Error{BISP_EINVAL, "mas"};
    if (n < 0 || (n > 0 && (!xyz || !keys_out || !order_out))) throw Error{BISP_EINVAL, "bad pointers or size"};
    if (n > kMaxParticles)
      throw Error{BISP_EINVAL, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                   std::to_string(kMaxParticles) + " particles"};
    if (n == 0) return BISP_OK;
    int st = BISP_OK;
    unsigned char* base = static_cast<unsigned char*>(scratch_address(&st));
    if (st != BISP_OK) throw Error{st, "cannot resolve the scratch array of bisp_cell_order_noalloc"};
    unsigned char* const start = base;
    cudaStream_t s = (cudaStream_t)stream;
    // carve the array: all offsets are multiples of 256 bytes
    auto take = [&](size_t bytes) {
      unsigned char* p = base;
      base += (bytes + 255) / 256 * 256;
      return p;
    };
    uint32_t* keys = reinterpret_cast<uint32_t*>(take((size_t)n * 4));
    uint32_t* idx = reinterpret_cast<uint32_t*>(take((size_t)n * 4));
    float4* frac = reinterpret_cast<float4*>(take((size_t)n * 16));
    double* part = reinterpret_cast<double*>(take((size_t)prep_blocks(n) * 8));
    int* bad = reinterpret_cast<int*>(take(256));
    float* ynorm = reinterpret_cast<float*>(take((BISP_LMAX + 1) * (BISP_LMAX + 1) * sizeof(float)));
    const size_t sortb = radix_sort_scratch_bytes(n);
    void* sortscr = take(sortb);
    if ((size_t)(base - start) > kScratchBytes) throw Error{BISP_ENOMEM, "no-allocation scratch layout overflow"};
    // the counter must start at zero; the table holds ones (no harmonics are needed here)
    BISP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    static const std::vector<float> ones((BISP_LMAX + 1) * (BISP_LMAX + 1), 1.f);
    BISP_CUDA(cudaMemcpyAsync(ynorm, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    PrepArgs a{};
    a.xyz = xyz;
    a.n = n;
    a.N = nmesh;
    a.H = box_len / nmesh;
    a.box = box_len;
    a.mas = mas;
    a.nchan = 0;
    a.keys = keys;
    a.idx = idx;
    a.frac = frac;
    a.vals = nullptr;
    a.partials = part;
    a.nsum = 1;
    a.bad = bad;
    a.ynorm = ynorm;
    launch_prep(a, s);
    int nbad = 0;
    BISP_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BISP_CUDA(cudaStreamSynchronize(s));
    if (nbad) throw Error{BISP_EINVAL, std::to_string(nbad) + " particles have non-finite or out-of-box positions"};
    int bits = 0;
    while ((1LL << bits) < (int64_t)nmesh * nmesh * nmesh) ++bits;
    radix_sort(keys, idx, keys_out, order_out, n, bits, sortscr, s, nullptr);
    BISP_CUDA(cudaStreamSynchronize(s));
    return BISP_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return (bisp_status)e.status;
  } catch (const std::exception& e) {  // nothing may leave the C ABI
    set_last_error(std::string("bisp_cell_order_noalloc: ") + e.what());
    return BISP_ECUDA;
  } catch (...) {
    set_last_error("bisp_cell_order_noalloc: unexpected exception");
    return BISP_ECUDA;
  }
}
