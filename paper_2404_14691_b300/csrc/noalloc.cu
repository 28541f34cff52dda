// sage_invoke_noalloc: one invocation of the function for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync are off
// limits -- a host thread that must never touch the device allocator (for
// example one that sits in a latency-critical loop, or inside a memory-budgeted
// runtime that hands out no allocations), or a caller that owns every byte of
// device memory itself and only lends this library the function's read-only
// data and the invocation's buffers.  sage_invoke needs a prepared sage_fn,
// whose workspace the pool allocates; this variant needs none.
//
// Where its scratch lives: the activations of the chain (bottom hidden layers,
// the concat buffer, top hidden layers) and the kernels' error word sit in one
// file-scope __device__ array of kScratchBytes.  Every GPU that loads this
// library holds that array until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a stand-in), so the
// first call on each device looks the address up with cudaGetSymbolAddress,
// with that device current, and caches it; make that first call before any
// stream capture.  The cached address belongs to the device's context as it was
// then: resetting the device (cudaDeviceReset) after the first call is not
// supported.  All calls share the one array: a call overwrites the last call's
// contents, and two calls whose kernels overlap on the GPU race.
//
// Errors the kernels find (a bag row outside its table, skipped; a tensor-core
// GEMM's bounded wait that ran out) land in the array's error word, which every
// call clears first; sage_noalloc_check reads it back and clears it.
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "../../include/sage.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr size_t kErrBytes = 256;                    // error word, cleared by every call

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[sage::kMaxDevices] = {};

sage_status noalloc_fail(sage_status st, const char* msg) {
  sage::set_last_error(msg);
  return st;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// The scratch address of the current device, looked up (once per device, with
// that device current) on first use.  *dev receives the device ordinal.
sage_status scratch_base(char** out, int* dev_out) {
  char msg[160];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= sage::kMaxDevices)
    return noalloc_fail(SAGE_ERR_CUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return noalloc_fail(SAGE_ERR_CUDA, msg);
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_scratch_ptr[dev]);
  if (dev_out) *dev_out = dev;
  return SAGE_OK;
}

}  // namespace

extern "C" sage_status sage_invoke_noalloc(const sage_fn_desc* shape, const void* tables, const void* weights,
                                           const sage_invocation* inv, void* stream_) {
  using namespace sage;
  char msg[256];
  if (!shape || !tables || !weights || !inv) return noalloc_fail(SAGE_ERR_INVALID, "null argument");
  const sage_fn_desc& d = *shape;
  if (d.dtype != SAGE_F32 && d.dtype != SAGE_BF16) return noalloc_fail(SAGE_ERR_INVALID, "bad dtype");
  if (d.num_tables < 1 || d.num_tables > kMaxTables || !d.rows)
    return noalloc_fail(SAGE_ERR_INVALID, "bad num_tables");
  const size_t es = d.dtype == SAGE_BF16 ? 2 : 4;
  const size_t rb = static_cast<size_t>(d.dim) * es;
  if (d.dim < 1 || rb < 16 || rb > 1024 || (rb & (rb - 1)))
    return noalloc_fail(SAGE_ERR_INVALID, "dim*elem must be a power of two in [16, 1024] bytes");
  if (d.n_dense < 1 || d.n_dense > 64 || d.n_bot < 1 || d.n_bot > 8 || d.n_top < 1 || d.n_top > 8 ||
      !d.bot_dims || !d.top_dims || d.top_dims[d.n_top - 1] != 1)
    return noalloc_fail(SAGE_ERR_INVALID, "bad layer shape");
  for (int t = 0; t < d.num_tables; ++t)
    if (d.rows[t] < 1 || d.rows[t] >= (int64_t(1) << 31)) return noalloc_fail(SAGE_ERR_INVALID, "bad rows");
  const int B = inv->batch;
  if (B < 0) return noalloc_fail(SAGE_ERR_INVALID, "negative batch");
  if (B == 0) return SAGE_OK;
  if (!inv->dense || !inv->indices || !inv->offsets || !inv->out)
    return noalloc_fail(SAGE_ERR_INVALID, "null invocation buffer");
  // the kernels read table rows and weights with 16-byte loads and TMA (weight
  // offsets are 256-byte aligned relative to the item), dense rows and outputs
  // with vector accesses: a misaligned buffer is refused here, before any launch
  if (!aligned(tables, 256) || !aligned(weights, 256))
    return noalloc_fail(SAGE_ERR_INVALID, "tables and weights must be 256-byte aligned");
  if (!aligned(inv->dense, 16) || !aligned(inv->out, 16))
    return noalloc_fail(SAGE_ERR_INVALID, "dense and out must be 16-byte aligned");
  if (!aligned(inv->indices, 4) || !aligned(inv->offsets, 8))
    return noalloc_fail(SAGE_ERR_INVALID, "indices must be 4-byte and offsets 8-byte aligned");

  // layers (in, out) and their places inside the weights item
  const int nb = d.n_bot, nt = d.n_top;
  const int cd = d.num_tables * d.dim + d.bot_dims[nb - 1];
  int lin[16], lout[16];
  int prev = d.n_dense;
  for (int l = 0; l < nb; ++l) {
    lin[l] = prev;
    lout[l] = d.bot_dims[l];
    prev = d.bot_dims[l];
  }
  prev = cd;
  for (int l = 0; l < nt; ++l) {
    lin[nb + l] = prev;
    lout[nb + l] = d.top_dims[l];
    prev = d.top_dims[l];
  }
  const void* W[16];
  const float* bias[16];
  size_t o = 0;
  for (int l = 0; l < nb + nt; ++l) {
    if (lin[l] < 1 || lout[l] < 1) return noalloc_fail(SAGE_ERR_INVALID, "bad layer shape");
    if (l >= 1 && l + 1 < nb + nt) {
      if (d.dtype == SAGE_BF16 && ((lin[l] % 64) || (lout[l] % 64)))
        return noalloc_fail(SAGE_ERR_INVALID, "bf16 hidden layers need multiples of 64");
      if (d.dtype == SAGE_F32 && ((lin[l] % 4) || (lout[l] % 4)))
        return noalloc_fail(SAGE_ERR_INVALID, "fp32 hidden layers need multiples of 4");
    }
    o = a256(o);
    W[l] = static_cast<const char*>(weights) + o;
    o += static_cast<size_t>(lin[l]) * lout[l] * es;
    o = a256(o);
    bias[l] = reinterpret_cast<const float*>(static_cast<const char*>(weights) + o);
    o += static_cast<size_t>(lout[l]) * 4;
  }

  // scratch layout for this batch: error word | bottom hidden | concat | top hidden
  size_t need = kErrBytes;
  for (int l = 0; l + 1 < nb; ++l) need += a256(static_cast<size_t>(B) * lout[l] * es);
  need += a256(static_cast<size_t>(B) * cd * es);
  for (int l = 0; l + 1 < nt; ++l) need += a256(static_cast<size_t>(B) * lout[nb + l] * es);
  if (need > kScratchBytes) {
    snprintf(msg, sizeof(msg), "batch of %d needs %zu bytes of scratch; the no-alloc scratch holds %zu bytes", B,
             need, kScratchBytes);
    return noalloc_fail(SAGE_ERR_INVALID, msg);
  }

  // per-device set-up: the array's device address, looked up with the device current
  char* base = nullptr;
  if (sage_status st = scratch_base(&base, nullptr); st != SAGE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  int* err = reinterpret_cast<int*>(base);
  if (cudaMemsetAsync(err, 0, kErrBytes, s) != cudaSuccess) return noalloc_fail(SAGE_ERR_CUDA, "memset");
  char* p = base + kErrBytes;
  char* bot[8];
  for (int l = 0; l + 1 < nb; ++l) {
    bot[l] = p;
    p += a256(static_cast<size_t>(B) * lout[l] * es);
  }
  char* concat = p;
  p += a256(static_cast<size_t>(B) * cd * es);
  char* top[8];
  for (int l = 0; l + 1 < nt; ++l) {
    top[l] = p;
    p += a256(static_cast<size_t>(B) * lout[nb + l] * es);
  }

  InvTable tab;
  tab.n = 1;
  tab.M = B;
  tab.d[0] = InvDesc{inv->dense, inv->indices, inv->offsets, inv->out, B, 0, inv->num_indices};
  cudaError_t e = cudaSuccess;
  char* bot_out = concat + static_cast<size_t>(d.num_tables) * d.dim * es;
  // bottom MLP
  e = launch_bottom0(d.dtype, tab, lin[0], lout[0], W[0], bias[0], nb == 1 ? bot_out : bot[0],
                     nb == 1 ? cd : lout[0], s);
  for (int l = 1; l < nb && e == cudaSuccess; ++l) {
    void* y = l == nb - 1 ? bot_out : bot[l];
    const int ldy = l == nb - 1 ? cd : lout[l];
    e = d.dtype == SAGE_BF16
            ? launch_linear_bf16_tc(B, lout[l], lin[l], bot[l - 1], lin[l], W[l], bias[l], 1, y, ldy, err, s)
            : launch_linear_f32(B, lout[l], lin[l], reinterpret_cast<const float*>(bot[l - 1]), lin[l],
                                static_cast<const float*>(W[l]), bias[l], 1, static_cast<float*>(y), ldy, s);
  }
  // gather into the concat columns [0, T*dim)
  if (e == cudaSuccess) {
    GatherArgs a;
    a.dtype = d.dtype;
    a.tables = static_cast<const char*>(tables);
    int64_t off = 0;
    for (int t = 0; t < d.num_tables; ++t) {
      a.table_off[t] = off;
      a.table_rows[t] = static_cast<int32_t>(d.rows[t]);
      off += d.rows[t] * static_cast<int64_t>(rb);
    }
    a.T = d.num_tables;
    a.dim = d.dim;
    a.out = concat;
    a.ldo = cd;
    a.err = err;
    e = launch_gather(a, tab, s);
  }
  // top MLP hidden layers and the head
  const char* x = concat;
  int ldx = cd;
  for (int l = 0; l + 1 < nt && e == cudaSuccess; ++l) {
    const int L = nb + l;
    e = d.dtype == SAGE_BF16
            ? launch_linear_bf16_tc(B, lout[L], lin[L], x, ldx, W[L], bias[L], 1, top[l], lout[L], err, s)
            : launch_linear_f32(B, lout[L], lin[L], reinterpret_cast<const float*>(x), ldx,
                                static_cast<const float*>(W[L]), bias[L], 1, reinterpret_cast<float*>(top[l]),
                                lout[L], s);
    x = top[l];
    ldx = lout[L];
  }
  if (e == cudaSuccess) {
    const int H = nb + nt - 1;
    e = launch_head(d.dtype, tab, lin[H], x, ldx, W[H], bias[H], s);
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "kernel launch: %s", cudaGetErrorString(e));
    return noalloc_fail(e == cudaErrorInvalidValue ? SAGE_ERR_INVALID : SAGE_ERR_CUDA, msg);
  }
  return SAGE_OK;
}

extern "C" sage_status sage_noalloc_check(void* stream_) {
  char* base = nullptr;
  if (sage_status st = scratch_base(&base, nullptr); st != SAGE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  int w = 0;
  // a plain copy into a host int and a memset: no allocation
  if (cudaMemcpyAsync(&w, base, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(base, 0, sizeof(int), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return noalloc_fail(SAGE_ERR_CUDA, "reading the no-alloc error word failed");
  if (w & sage::kErrTimeout) return noalloc_fail(SAGE_ERR_DEVICE, "a kernel's bounded wait ran out");
  if (w & sage::kErrBounds) return noalloc_fail(SAGE_ERR_BOUNDS, "a bag row index was outside its table");
  return SAGE_OK;
}
