// Host-side launch interface of the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "common.cuh"
#include "../../include/sage.h"

namespace sage {

// Sets the thread-local message that sage_last_error() returns.
void set_last_error(const char* msg);

// Asynchronous fused batch from host buffers on a chosen workspace slot (-1: next in turn).
sage_status host_batch_async(sage_fn f, const sage_host_invocation* invs, int n, cudaStream_t s, int slot);

// A host invocation's bags lie inside its indices: offsets[0] == 0, the offsets
// never decrease, and offsets[T * B] == num_indices (an empty batch passes).  Both
// host entry points check this before any copy, so a malformed request is refused
// instead of reading outside the indices it copied.
bool host_csr_valid(const sage_host_invocation& v, int T);

// Kernels launched by this library so far (all pools, all threads).
void count_launch(int n = 1);
int64_t launches();

// Kernel function attributes (shared-memory size, carve-out) are set per device:
// a launcher runs its set-up once on every device that uses it, from any thread.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
  std::atomic<uint64_t> done{0};
  std::mutex mu;
};
// Runs init(dev) the first time the current device reaches this DeviceOnce; *dev
// (optional) receives the current device.  init's error is returned and the set-up
// is retried on the next call.
template <class F>
cudaError_t device_once(DeviceOnce& o, F&& init, int* dev_out = nullptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (dev_out) *dev_out = dev;
  const uint64_t bit = uint64_t(1) << dev;
  if (o.done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  std::lock_guard<std::mutex> g(o.mu);
  if (o.done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  const cudaError_t e = init(dev);
  if (e == cudaSuccess) o.done.fetch_or(bit, std::memory_order_release);
  return e;
}
// SMs of the current device (looked up once per device).
int device_sms();

// Embedding-bag sum over a fused batch (the gather of the function).
struct GatherArgs {
  int dtype;                         // 0 fp32 tables/out, 1 bf16 tables/out
  const char* tables;                // tables item
  int64_t table_off[kMaxTables];     // byte offset of table t in the item
  int32_t table_rows[kMaxTables];
  int T;
  int dim;
  void* out;                         // [M, ldo] elements of the table dtype
  int ldo;
  int* err;
  float* out_lo = nullptr;           // fp32 only, optional: out becomes the tf32 hi plane, out_lo the residual
  // optional: two counters {next, done}, zero before the launch and zero again after it
  // (the last block to finish resets them); with them, warps claim their bags (or runs
  // of bags) one group at a time instead of a fixed grid-stride share, so blocks that
  // start early -- beside another kernel that holds part of the GPU -- take more work
  unsigned* work = nullptr;
};
cudaError_t launch_gather(const GatherArgs& a, const InvTable& tab, cudaStream_t s);

// Bottom layer 0: y = ReLU(dense W0^T + b0) with the dense rows read from each
// invocation of the batch.  W0 [N, K] in the dtype, y [M, ldy] in the dtype.
cudaError_t launch_bottom0(int dtype, const InvTable& tab, int K, int N, const void* W, const float* bias,
                           void* y, int ldy, cudaStream_t s, float* y_lo = nullptr);

// Head: out_i[b] = sigmoid(h[r, :] . w + c) for every row r of the batch, written
// to its invocation's out.  h [M, ldh] in the dtype, w [K] in the dtype, c fp32.
cudaError_t launch_head(int dtype, const InvTable& tab, int K, const void* h, int ldh, const void* w,
                        const float* c, cudaStream_t s, const float* h_lo = nullptr);

// 2-D TMA tensor map of a row-major matrix [rows, cols] (row stride ld elements;
// dtype 0 fp32, 1 bf16), boxes of box_rows x box_cols, 128-byte swizzle, zero
// fill outside the matrix.
bool make_tmap_2d(CUtensorMap* m, int dtype, const void* base, int rows, int cols, int ld, int box_cols,
                  int box_rows);

// Tile configuration of a tensor-core GEMM launch: N tile and pipeline depth;
// {0, 0} lets the launcher choose by its shape heuristic.
struct GemmCfg {
  int bn;
  int stages;
};
enum : int { kGemmBf16 = 1, kGemmTf32x3 = 2, kGemmTf32Pre = 3, kBottom01 = 4, kGatherTop0 = 5 };
int gemm_candidates(int kind, GemmCfg* out, int max);
int tf32_candidates(GemmCfg* out, int max);
int tf32_presplit_candidates(GemmCfg* out, int max);
// Tuned configuration for a GEMM shape ({0, 0} if none was tuned).
GemmCfg tuned_gemm(int kind, int M, int N, int K);
// Times every configuration of one shape and records the fastest.
sage_status autotune_gemm(int kind, int M, int N, int K, cudaStream_t s, GemmCfg* chosen, double* best_ms);
// Fused bottom layers 0 and 1 (and 2, when N2 > 0 and the shape allows) against the
// separate kernels (kBottom01).
sage_status autotune_bottom01(int M, int K0, int N0, int N1, int N2, cudaStream_t s, GemmCfg* chosen);

// Dense layers y = act(x W^T + b).
cudaError_t launch_linear_f32(int M, int N, int K, const float* x, int ldx, const float* W, const float* bias,
                              int relu, float* y, int ldy, cudaStream_t s);
cudaError_t launch_linear_bf16_tc(int M, int N, int K, const void* x, int ldx, const void* W,
                                  const float* bias, int relu, void* y, int ldy, int* err, cudaStream_t s,
                                  GemmCfg cfg = GemmCfg{0, 0});
// fp32 layer on the tensor cores from pre-split hi/lo planes of x and W; writes
// its output as hi/lo planes.
cudaError_t launch_linear_f32_tc_presplit(int M, int N, int K, const float* xh, const float* xl, int ldx,
                                          const float* wh, const float* wl, const float* bias, int relu, float* yh,
                                          float* yl, int ldy, int* err, cudaStream_t s, GemmCfg cfg = GemmCfg{0, 0});
// True when the last hidden layer (N outputs) can fuse the sigmoid head with tile
// configuration cfg: a persistent configuration and N / 64 a power of two.
inline bool head_fusable(GemmCfg cfg, int N) {
  const int G = N / 64;
  return cfg.stages >= 100 && cfg.bn > 0 && N % 64 == 0 && N % cfg.bn == 0 && G > 0 && (G & (G - 1)) == 0;
}
// The last hidden layer with the head fused (hp); writes no Y.
cudaError_t launch_linear_f32_tc_presplit_head(int M, int N, int K, const float* xh, const float* xl, int ldx,
                                               const float* wh, const float* wl, const float* bias, int relu,
                                               int* err, cudaStream_t s, GemmCfg cfg, const HeadParams& hp);
cudaError_t launch_linear_bf16_tc_head(int M, int N, int K, const void* x, int ldx, const void* W,
                                       const float* bias, int relu, int* err, cudaStream_t s, GemmCfg cfg,
                                       const HeadParams& hp);
// Bottom layers 0 and 1 of a pre-split fp32 function in one kernel: layer 0
// (K0 <= 15 dense inputs, N0 outputs, ReLU) is computed into layer 1's shared-memory
// A tiles; layer 1's output (N1 columns, ReLU) is written as hi/lo planes.  With
// layer 2's weight planes and bias (N2 outputs) and configuration (256, 202) -- or
// {0, 0} when bottom012_fusable -- the kernel computes layer 2 as well and writes
// only its output (yh / yl / ldy then describe layer 2's output); *layers reports 2
// or 3.  Same bits as launch_bottom0 followed by launch_linear_f32_tc_presplit per
// layer.  cfg: one of bottom01_candidates' fused configurations, or {0, 0}.
bool bottom01_fusable(int K0, int N0, int N1);
// Layer 2 too: N1 = 256, N2 a multiple of 32 up to 256, one 128-row tile per SM.
bool bottom012_fusable(int N1, int N2, int M);
int bottom01_candidates(GemmCfg* out, int max);  // the last one, {1, 1}, means separate kernels
GemmCfg bottom01_default(int N1);
cudaError_t launch_bottom01_f32(const InvTable& tab, int K0, int N0, const float* W0, const float* b0, int N1,
                                const float* w1h, const float* w1l, const float* b1, float* yh, float* yl, int ldy,
                                int* err, cudaStream_t s, GemmCfg cfg, const float* w2h = nullptr,
                                const float* w2l = nullptr, const float* b2 = nullptr, int N2 = 0,
                                int* layers = nullptr);
// The gather and the first top layer of a pre-split fp32 function in one kernel:
// y = ReLU([pooled, bottom] W0^T + b0) as hi/lo planes, the pooled columns summed
// straight into the GEMM's shared-memory A tiles (never written), the bottom
// output's columns read from x (hi/lo planes of the concat buffer, row stride ldx,
// written before the launch).  Tables of 64 fp32 columns; N0 = 256 or 512; K0 =
// T * 64 + the bottom output's width (a multiple of 32).  Same bits as
// launch_gather followed by launch_linear_f32_tc_presplit.
bool gather_top0_fusable(int dtype, int dim, int T, int n_bot_out, int N0, bool presplit);
cudaError_t launch_gather_top0_f32(const GatherArgs& a, const InvTable& tab, int N0, int K0, const float* xh,
                                   const float* xl, int ldx, const float* wh, const float* wl, const float* b0,
                                   float* yh, float* yl, int ldy, int* err, cudaStream_t s);
void preload_gather_top0_kernels();
// hi[i] = tf32(src[i]) (round to nearest), lo[i] = src[i] - hi[i].
cudaError_t launch_split_planes(const float* src, float* hi, float* lo, size_t n, cudaStream_t s);
// fp32 layer on the tensor cores: three tf32 products of the hi/lo split of x and W.
cudaError_t launch_linear_f32_tc(int M, int N, int K, const float* x, int ldx, const float* W, const float* bias,
                                 int relu, float* y, int ldy, int* err, cudaStream_t s, GemmCfg cfg = GemmCfg{0, 0});

// Kernel loading: query every kernel of a translation unit once, which makes the
// CUDA runtime load its module (lazy loading defers this to first use).
void preload_gather_kernels();
void preload_simt_kernels();
void preload_tc_kernels();
void preload_tf32_kernels();
void preload_bottom01_kernels();

// ---------------------------------------------------------------- cross-process sharing
//
// The read-only copy of a function can live in one process (the owner, whose pool
// was created exportable) and be mapped by others (Sec. 5.1: the data is prepared
// by a daemon process while the function process sets up its own context).  The
// owner allocates that copy as virtual-memory-management (VMM) physical memory
// that can be exported as a POSIX file descriptor; a client imports the
// descriptor and maps the same physical memory into its own address space.

// One exportable device allocation: physical handle, its mapping here, mapped size
// (a multiple of the allocation granularity).
struct VmmBlock {
  unsigned long long handle = 0;  // CUmemGenericAllocationHandle
  void* va = nullptr;
  size_t size = 0;
};
// Allocates >= bytes of exportable device memory on `device`, mapped read-write in
// this process.  false (and a last-error message) on failure.
bool vmm_alloc(int device, size_t bytes, VmmBlock* out);
// Unmaps and releases this process's reference (the physical memory lives on while
// another process still maps it).
void vmm_free(VmmBlock& b);

// A function's read-only data mapped from another process.  The client pool owns
// it through the entry it backs and destroys it after the entry's last use.
struct ImportedData {
  char* tables = nullptr;
  char* weights = nullptr;
  // Blocks until the owner reports the data complete (true) or failed / the link
  // closed (false).
  virtual bool wait_ready() = 0;
  // Makes a blocked wait_ready() return false (called before the entry is freed).
  virtual void interrupt() = 0;
  virtual ~ImportedData() {}
};

// ---------------------------------------------------------------- SM partitions

// Green contexts splitting the SMs into groups; streams created in a group run
// their kernels on its SMs only.
struct Partition {
  struct Group {
    CUgreenCtx ctx = nullptr;
    int sms = 0;
    std::vector<CUstream> streams;
  };
  int device = 0;
  int total_sms = 0;
  std::vector<Group> groups;
  // n groups of min_sms SMs (rounded up to the hardware granularity) or, with
  // min_sms = 0, of SMs / n rounded down to it.
  static sage_status create(int device, int n, int min_sms, Partition** out);
  // A new non-blocking stream in group i (destroyed with the partition).
  sage_status stream(int i, cudaStream_t* out);
  ~Partition();
};
// True when s belongs to a green context: launch chains on it stay on it (no
// branch stream, no graph of the primary context).
bool stream_is_confined(cudaStream_t s);

// Shape checks of a descriptor without its data sources (the attaching side has none).
sage_status check_shape(const sage_fn_desc* d);
// The shape signature two sides compare before one maps the other's copy.
std::string shape_signature(const sage_fn_desc* d);
// Prepares `shape` in `pool` on data another process owns: like sage_prepare but
// the read-only items are `imp`'s mappings and "staging" is waiting for the owner.
// Takes ownership of imp (also on failure).
sage_status prepare_imported(sage_pool pool, const sage_fn_desc* shape, ImportedData* imp, sage_fn* out);
// The pool's CUDA ordinal, and whether it allocates exportable read-only items.
int pool_device(sage_pool pool);
bool pool_exportable(sage_pool pool);
// The exportable blocks holding f's tables and weights (the owner's side).
sage_status fn_export(sage_fn f, VmmBlock* tables, VmmBlock* weights);

}  // namespace sage
