// noalloc_sort.cuh — cvetl_sort_u64_noalloc: the library's stable LSD radix sort of 64-bit
// keys, with every byte of its scratch memory (ping-pong keys and values, look-back status,
// digit histograms, tile counters, error word) in one file-scope device array instead of
// cudaMalloc'ed buffers. The caller passes the input keys and the output arrays.
//
// Who needs this: callers that may not allocate device memory themselves — code running
// inside a host framework that owns the device memory pool and forbids side allocations,
// and latency-critical loops in which a cudaMalloc / cudaFree (which can synchronise the
// device) would stall the pipeline. It is a fixed-size service: at most
// CVETL_NOALLOC_MAX_PAIRS keys per call.
#pragma once
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "radix_sort.cuh"

namespace cvetl {
namespace noalloc {

constexpr uint32_t kMaxPairs = CVETL_NOALLOC_MAX_PAIRS;
constexpr uint32_t kMaxTiles = (kMaxPairs + rs::kTile - 1) / rs::kTile;
// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t kOffKeys = 0;                                        // u64 x kMaxPairs
constexpr size_t kOffVals = kOffKeys + 8ull * kMaxPairs;              // u32 x kMaxPairs
constexpr size_t kOffStatus = kOffVals + 4ull * kMaxPairs;            // u32 x kMaxTiles x 256
constexpr size_t kOffHist = kOffStatus + 4ull * kMaxTiles * rs::kRadix;  // u32 x 8 x 256
constexpr size_t kOffTiles = kOffHist + 4ull * rs::kMaxPasses * rs::kRadix;  // u32 x 8
constexpr size_t kOffErr = kOffTiles + 256;                           // u32
constexpr size_t kBytes = kOffErr + 256;
static_assert(kOffVals % 256 == 0 && kOffStatus % 256 == 0 && kOffHist % 256 == 0, "alignment");

constexpr int kMaxDevices = 64;
// device address of the array, per device (null until that device's set-up); published with
// release order after the set-up, read with acquire order, so a thread that sees the address
// also sees the kernel attribute set before it
static std::atomic<void*> g_scratch_addr[kMaxDevices];
static std::mutex g_setup_mutex;

}  // namespace noalloc
}  // namespace cvetl

// The scratch itself: one array per device that loads the library, held until the process
// exits. In host code this name is only a stand-in; kernels get the device address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_cvetl_noalloc_scratch[cvetl::noalloc::kBytes];

extern "C" cvetl_status cvetl_sort_u64_noalloc(const uint64_t* keys_in, uint64_t* keys_out,
                                               uint32_t* perm_out, int64_t n, int32_t begin_bit,
                                               int32_t end_bit, void* stream) {
  using namespace cvetl;
  using namespace cvetl::noalloc;
  cvetl_ctx* c = nullptr;  // errors go to cvetl_last_error(NULL)
  if (n < 0 || n > (int64_t)kMaxPairs)
    return fail(c, CVETL_EINVAL, "cvetl_sort_u64_noalloc: n = %lld is outside [0, %u] (CVETL_NOALLOC_MAX_PAIRS)",
                (long long)n, kMaxPairs);
  if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit)
    return fail(c, CVETL_EINVAL, "cvetl_sort_u64_noalloc: bit range [%d, %d) is not inside [0, 64)",
                begin_bit, end_bit);
  if (n == 0) return CVETL_OK;
  if (!keys_in || !keys_out || !perm_out)
    return fail(c, CVETL_EINVAL, "cvetl_sort_u64_noalloc: NULL array");
  if ((const void*)keys_in == (const void*)keys_out)
    return fail(c, CVETL_EINVAL, "cvetl_sort_u64_noalloc: keys_out must not be keys_in");
  cudaStream_t st = (cudaStream_t)stream;
  {
    // the call ends with a read-back of the device error word and a stream synchronisation,
    // which a stream capture does not allow: refuse instead of invalidating the caller's graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(c, CVETL_ESTATE, "cvetl_sort_u64_noalloc: the stream is capturing; this call cannot be captured");
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(c, CVETL_EINVAL, "cvetl_sort_u64_noalloc: device %d beyond the supported %d", dev, kMaxDevices);
  // Set-up, once per device, with that device current: the array's device address and the
  // kernel's shared-memory limit. This happens inside the first call on each device.
  void* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_cvetl_noalloc_scratch));
      CK(cudaFuncSetAttribute(rs::k_onesweep<unsigned long long>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, rs::kTile * 12));
      g_scratch_addr[dev].store(p, std::memory_order_release);
      addr = p;
    }
  }
  unsigned char* base = (unsigned char*)addr;
  unsigned long long* s_keys = (unsigned long long*)(base + kOffKeys);
  uint32_t* s_vals = (uint32_t*)(base + kOffVals);
  uint32_t* status = (uint32_t*)(base + kOffStatus);
  uint32_t* hist = (uint32_t*)(base + kOffHist);
  uint32_t* tiles = (uint32_t*)(base + kOffTiles);
  uint32_t* err = (uint32_t*)(base + kOffErr);

  const uint32_t un = (uint32_t)n;
  const int passes = (end_bit - begin_bit + rs::kBits - 1) / rs::kBits;
  const uint32_t ntiles = (un + rs::kTile - 1) / rs::kTile;
  // the array keeps the previous call's contents: clear what must start at zero
  CK(cudaMemsetAsync(hist, 0, 4ull * rs::kMaxPasses * rs::kRadix, st));
  CK(cudaMemsetAsync(tiles, 0, 4ull * rs::kMaxPasses, st));
  CK(cudaMemsetAsync(err, 0, 4, st));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int hb = (int)((un + rs::kBlock - 1) / rs::kBlock);
  if (hb > sms * 4) hb = sms * 4;
  rs::k_histogram<unsigned long long><<<hb, rs::kBlock, 0, st>>>(
      (const unsigned long long*)keys_in, un, begin_bit, passes, end_bit, hist, nullptr);
  rs::k_hist_scan<<<passes, rs::kBlock, 0, st>>>(hist);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, CVETL_ECUDA, "cvetl_sort_u64_noalloc: %s", cudaGetErrorString(e));
  }
  // Ping-pong between the caller's outputs and the scratch so that the last pass lands in
  // the outputs: with an odd pass count pass 0 writes the outputs, else the scratch.
  const unsigned long long* kin = (const unsigned long long*)keys_in;
  const uint32_t* vin = nullptr;  // first pass: value = input position
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    unsigned long long* kout = to_out ? (unsigned long long*)keys_out : s_keys;
    uint32_t* vout = to_out ? perm_out : s_vals;
    CK(cudaMemsetAsync(status, 0, 4ull * ntiles * rs::kRadix, st));
    rs::k_onesweep<unsigned long long><<<ntiles, rs::kBlock, (size_t)rs::kTile * 12, st>>>(
        kin, vin, kout, vout, un, begin_bit + rs::kBits * p,
        rs::digit_mask(begin_bit + rs::kBits * p, end_bit), hist + p * rs::kRadix, status,
        tiles + p, err, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, CVETL_ECUDA, "cvetl_sort_u64_noalloc: %s", cudaGetErrorString(e));
    kin = kout;
    vin = vout;
  }
  uint32_t herr = 0;
  CK(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr & kErrLookbackTimeout)
    return fail(c, CVETL_ETIMEOUT, "cvetl_sort_u64_noalloc: a look-back wait gave up");
  return CVETL_OK;
}
