// Device helpers shared by the sm_103a kernels: bf16 packing, bounded mbarrier
// waits, TMA tile loads and tcgen05 (5th-generation tensor core) wrappers in
// inline PTX.  Host code includes this header only for the launch descriptors.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace sage {

// Per-kernel error bits written to the caller's device error word.
enum : int { kErrBounds = 1, kErrTimeout = 2 };

// Upper limit on the invocations fused into one launch (they travel in the
// kernel parameter block, so no descriptor copy precedes a batch).
constexpr int kMaxInv = 256;
constexpr int kMaxTables = 128;

// One invocation of a fused batch: its samples are rows [row_base, row_base+batch)
// of the batch's activations.
struct InvDesc {
  const float* dense;      // [batch, n_dense]
  const int32_t* indices;
  const int64_t* offsets;  // [T*batch + 1]
  float* out;              // [batch]
  int batch;
  int row_base;
  int64_t nidx;            // indices of the invocation if known on the host (cost model only), else 0
};

constexpr int kInvBlocks = 1024;

struct InvTable {
  int n;                   // invocations
  int M;                   // total rows
  InvDesc d[kMaxInv];
  // coarse index for n > 1: blk[k] = the invocation owning row k << blk_shift
  // (index_invocations fills it on the host)
  int blk_shift;
  uint8_t blk[kInvBlocks];
};

// Fill the coarse index of a table whose n, M and row bases are set.
inline void index_invocations(InvTable& t) {
  int shift = 0;
  while (t.M > 0 && ((t.M - 1) >> shift) >= kInvBlocks) ++shift;
  t.blk_shift = shift;
  const int nb = t.M > 0 ? ((t.M - 1) >> shift) + 1 : 0;
  int i = 0;
  for (int k = 0; k < nb; ++k) {
    while (i + 1 < t.n && t.d[i + 1].row_base <= (k << shift)) ++i;
    t.blk[k] = static_cast<uint8_t>(i);
  }
}

// Index of the invocation owning packed row r (row_base ascending, n > 1): the
// coarse index's invocation for r's block, then forward over the invocations that
// start inside the block.
__device__ __forceinline__ int find_inv(const InvTable& tab, int r) {
  int i = tab.blk[r >> tab.blk_shift];
  while (i + 1 < tab.n && tab.d[i + 1].row_base <= r) ++i;
  return i;
}

// ---------------------------------------------------------------- head order
//
// The sigmoid head z = h . w + c is summed in one fixed order, shared by the head
// kernel and by the GEMM epilogue that fuses it, so both give the same bits:
// products h_k w_k in 32-column chunks (zero beyond K) are added by a butterfly
// tree (pairs 16 apart, then 8, 4, 2, 1 -- what an xor-shuffle reduction gives in
// every lane); a 64-column group is chunk(2g) + chunk(2g+1); z = g_0 + g_1 + ...
// left to right, then + c.  Products and sums use __fmul_rn / __fadd_rn, which the
// compiler never contracts into FMAs, so both implementations round alike.
__device__ __forceinline__ float head_tree32(float (&p)[32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < o; ++i) p[i] = __fadd_rn(p[i], p[i + o]);
  return p[0];
}

__device__ __forceinline__ float head_sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

// The head fused into the epilogue of the last hidden layer (N outputs, N / 64 a
// power of two).  Each epilogue thread owns one row of a tile: it writes the row's
// 64-column group sums to part, then adds its group count to the row's arrival
// counter; the thread that completes the row's count (counters only grow, so
// "complete" is modulo N / 64) sums the groups and writes the sigmoid output.
struct HeadFuse {
  const void* w = nullptr;    // [N] head weights, the layer's dtype
  const float* c = nullptr;   // [1] head bias
  float* part = nullptr;      // [rows, N / 64] group sums
  unsigned* cnt = nullptr;    // [rows] arrival counters
};
struct HeadParams {
  HeadFuse f;
  InvTable tab;
};

__device__ __forceinline__ void head_write(const HeadParams& hp, int row, float z) {
  const int i = hp.tab.n == 1 ? 0 : find_inv(hp.tab, row);
  hp.tab.d[i].out[row - hp.tab.d[i].row_base] = head_sigmoid(__fadd_rn(z, hp.f.c[0]));
}

// Finish one row of the fused head from this tile's NG group sums gs (groups
// g0 .. g0+NG-1 of G).  A tile holding the whole row (NG == G) finishes it in
// registers; otherwise the sums go to part and the row's counter is bumped with
// one acquire-release atomic (it publishes these sums and, for the tile that
// completes the row, makes the other tiles' sums visible).
template <int NG>
__device__ __forceinline__ void head_row(const HeadParams& hp, int row, const float (&gs)[NG], unsigned g0,
                                         unsigned G) {
  if (NG == G) {
    float z = gs[0];
#pragma unroll
    for (int g = 1; g < NG; ++g) z = __fadd_rn(z, gs[g]);
    head_write(hp, row, z);
    return;
  }
  float* pr = hp.f.part + static_cast<size_t>(row) * G;
#pragma unroll
  for (int g = 0; g < NG; ++g) pr[g0 + g] = gs[g];
  unsigned prev;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;"
               : "=r"(prev)
               : "l"(hp.f.cnt + row), "r"(static_cast<unsigned>(NG))
               : "memory");
  if ((prev + NG) % G != 0) return;
  float z = __ldcg(pr);
  for (unsigned g = 1; g < G; ++g) z = __fadd_rn(z, __ldcg(pr + g));
  head_write(hp, row, z);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
  __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
  return __bfloat1622float2(v);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The first 1024-byte-aligned byte of a dynamic shared-memory buffer, reached by
// plain pointer arithmetic (no round trip through an integer), so the compiler
// still knows the pointer is shared and emits shared-memory loads and stores.
__device__ __forceinline__ uint8_t* smem_align1024(uint8_t* raw) {
  return raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
}

// ---------------------------------------------------------------- mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Gives up after about two
// seconds of %globaltimer (checked every 256 polls), sets kErrTimeout in *err and
// returns false, so that no kernel can spin forever.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull || i > (1u << 30)) {
        if (err) atomicOr(err, kErrTimeout);
        return false;
      }
    }
  }
}

// ---------------------------------------------------------------- TMA

// 2-D tiled bulk tensor load global -> shared, completion counted on `bar`.
// x is the innermost (contiguous) coordinate in elements.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tiled bulk tensor store shared -> global (rows outside the tensor map are
// not written), tracked as a bulk group of the issuing thread.
__device__ __forceinline__ void tma_store_2d(const void* tmap, const void* smem_src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tmap)),
               "r"(smem_u32(smem_src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Wait until all of this thread's bulk groups have completed their writes.
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Barrier over the `count` threads (a multiple of 32) that use barrier `id` (1..15).
__device__ __forceinline__ void named_barrier_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// ---------------------------------------------------------------- tcgen05

// Allocate `ncols` (power of two >= 32) tensor-memory columns; the whole warp
// executes this; the base address is written to *dst_smem.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte
// swizzle (rows of 128 B, 8-row atoms of 1024 B): start address, leading byte
// offset (unused for this layout, encoded 1), stride byte offset 1024 B between
// 8-row groups, descriptor version 1, layout type 2 = SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D fp32, A and B bf16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// Instruction descriptor of tcgen05.mma kind::tf32: D fp32, A and B tf32 (fp32
// bit patterns in shared memory), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same with the A operand kept in the tensor core's collector buffer for the
// next MMA (fill), or taken from it and released (lastuse): of two consecutive MMAs
// with the same A tile, the second reads no A from shared memory.
__device__ __forceinline__ void tc_mma_tf32_fill_a(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                                   uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_mma_tf32_lastuse_a(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                                      uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// fp32 -> nearest tf32 (ties away from zero), kept in an fp32 bit pattern.
__device__ __forceinline__ float to_tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Make this thread's generic-proxy shared-memory writes visible to the async
// proxy (TMA / tensor cores).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on `bar` when every tcgen05 operation issued so far by this
// thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Load 32 consecutive fp32 columns of this thread's TMEM lane (32x32b shape).
__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- tail epilogue
//
// Output of a persistent GEMM's last tile (per CTA) as tf32 hi / fp32 lo planes,
// y = act(acc + bias).  When that tile's MMAs have completed the CTA's stage ring
// is idle, so each epilogue warp stages its 32 rows x 32 columns there (128-byte
// swizzle: row r's 16-byte chunk j at r * 128 + ((j ^ r % 8) * 16), conflict-free)
// and writes them with TMA stores: whole 128-byte row pieces instead of a 16-byte
// piece of 32 different rows per store instruction.  The warp handles column
// blocks first, first + step, ... (32 columns each) of its 32 rows, so several
// warps can share one row quarter.  `stg` is the warp's NP hi/lo buffer pairs
// (8 KB each, 1024-byte aligned); `tm` its TMEM lanes at column 0; (x0, y0) the
// tile's first column and the quarter's first row in the output; `live` false
// when all 32 rows lie beyond the output (nothing is stored); `ncols` (<= BN, a
// multiple of 32) the tile's width.  Same arithmetic as the direct stores, so the
// same bits.
template <int BN, int NP>
__device__ __forceinline__ void tail_store_f32_planes(uint32_t tm, uint8_t* stg, int lane,
                                                      const float* __restrict__ bias, bool relu,
                                                      const void* tmYh, const void* tmYl, int x0, int y0,
                                                      bool live, int first = 0, int step = 1, int ncols = BN) {
  int it = 0;
#pragma unroll 1
  for (int c0 = 32 * first; c0 < ncols; c0 += 32 * step, ++it) {
    uint32_t v[32];
    tmem_ld_32cols(tm + c0, v);
    tmem_ld_wait();
    uint8_t* hb = stg + (it % NP) * 8192;
    uint8_t* lb = hb + 4096;
    if (it >= NP) {
      if (lane == 0) tma_store_wait_read<NP - 1>();  // this pair's stores of NP blocks ago
      __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        o[u] = __uint_as_float(v[4 * j + u]) + __ldg(bias + x0 + c0 + 4 * j + u);
        if (relu) o[u] = fmaxf(o[u], 0.f);
      }
      float4 h, l;
      h.x = to_tf32_rna(o[0]);
      h.y = to_tf32_rna(o[1]);
      h.z = to_tf32_rna(o[2]);
      h.w = to_tf32_rna(o[3]);
      l.x = o[0] - h.x;
      l.y = o[1] - h.y;
      l.z = o[2] - h.z;
      l.w = o[3] - h.w;
      const uint32_t off = static_cast<uint32_t>(lane * 128 + ((j ^ (lane & 7)) << 4));
      *reinterpret_cast<float4*>(hb + off) = h;
      *reinterpret_cast<float4*>(lb + off) = l;
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      if (live) {
        tma_store_2d(tmYh, hb, x0 + c0, y0);
        tma_store_2d(tmYl, lb, x0 + c0, y0);
      }
      tma_store_commit();
    }
  }
  if (lane == 0) tma_store_wait_all();
  __syncwarp();
}

}  // namespace sage
