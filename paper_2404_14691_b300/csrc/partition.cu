// SM partitions: streams whose kernels run on a fixed subset of the GPU's SMs
// (green contexts), so that functions served side by side do not take each
// other's SMs (the multi-function partitioning the paper lists among its
// lessons, Sec. 7.10).
//
// A partition splits the device's SM resource into equal groups (an equal share
// rounded down, an explicit size rounded up, to the hardware's partition
// granularity), creates one green context per group and
// streams inside it.  Kernels launched on such a stream through the runtime API
// run on the group's SMs only.  Launch chains on a confined stream stay on that
// stream: no branch stream of the primary context, no CUDA graph captured there.
#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/sage.h"
#include "kernels.h"

namespace sage {
namespace {

struct Green {
  decltype(&cuDeviceGet) device_get = nullptr;
  decltype(&cuDeviceGetDevResource) get_resource = nullptr;
  decltype(&cuDevSmResourceSplitByCount) split = nullptr;
  decltype(&cuDevResourceGenerateDesc) gen_desc = nullptr;
  decltype(&cuGreenCtxCreate) create = nullptr;
  decltype(&cuGreenCtxDestroy) destroy = nullptr;
  decltype(&cuGreenCtxStreamCreate) stream_create = nullptr;
  decltype(&cuStreamDestroy) stream_destroy = nullptr;
  decltype(&cuStreamGetCtx_v2) stream_ctx = nullptr;
  bool ok = false;
};

template <class F>
void entry(const char* name, F* out) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12050, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    *out = reinterpret_cast<F>(p);
}

const Green& green() {
  static Green g;
  static std::once_flag once;
  std::call_once(once, [] {
    entry("cuDeviceGet", &g.device_get);
    entry("cuDeviceGetDevResource", &g.get_resource);
    entry("cuDevSmResourceSplitByCount", &g.split);
    entry("cuDevResourceGenerateDesc", &g.gen_desc);
    entry("cuGreenCtxCreate", &g.create);
    entry("cuGreenCtxDestroy", &g.destroy);
    entry("cuGreenCtxStreamCreate", &g.stream_create);
    entry("cuStreamDestroy", &g.stream_destroy);
    entry("cuStreamGetCtx", &g.stream_ctx);
    g.ok = g.device_get && g.get_resource && g.split && g.gen_desc && g.create && g.destroy && g.stream_create &&
           g.stream_destroy && g.stream_ctx;
  });
  return g;
}

}  // namespace

bool stream_is_confined(cudaStream_t s) {
  if (!s) return false;
  const Green& g = green();
  if (!g.stream_ctx) return false;
  CUcontext c = nullptr;
  CUgreenCtx gc = nullptr;
  if (g.stream_ctx(reinterpret_cast<CUstream>(s), &c, &gc) != CUDA_SUCCESS) {
    cudaGetLastError();
    return false;
  }
  return gc != nullptr;
}

Partition::~Partition() {
  const Green& g = green();
  for (auto& grp : groups) {
    for (CUstream s : grp.streams) g.stream_destroy(s);
    if (grp.ctx) g.destroy(grp.ctx);
  }
}

sage_status Partition::create(int device, int n, int min_sms, Partition** out) {
  *out = nullptr;
  const Green& g = green();
  if (!g.ok) return set_last_error("green-context entry points unavailable"), SAGE_ERR_CUDA;
  if (n < 1) return set_last_error("need at least one group"), SAGE_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
    cudaGetLastError();
    return set_last_error("bad device"), SAGE_ERR_INVALID;
  }
  CUdevice dev = 0;
  if (g.device_get(&dev, device) != CUDA_SUCCESS) return set_last_error("cuDeviceGet failed"), SAGE_ERR_CUDA;
  CUdevResource all;
  if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS)
    return set_last_error("cuDeviceGetDevResource failed"), SAGE_ERR_CUDA;
  const int total = static_cast<int>(all.sm.smCount);
  const int gran = std::max<int>(1, std::max(all.sm.minSmPartitionSize, all.sm.smCoscheduledAlignment));
  // an explicit size rounds up to the granularity; an equal share rounds down
  int per = min_sms > 0 ? (min_sms + gran - 1) / gran * gran : total / n / gran * gran;
  if (per < static_cast<int>(all.sm.minSmPartitionSize)) per = static_cast<int>(all.sm.minSmPartitionSize);
  if (per * n > total)
    return set_last_error("the SMs cannot hold that many groups of that size"), SAGE_ERR_INVALID;
  std::vector<CUdevResource> res(n);
  unsigned int nb = static_cast<unsigned int>(n);
  CUdevResource rem;
  if (g.split(res.data(), &nb, &all, &rem, 0, static_cast<unsigned int>(per)) != CUDA_SUCCESS ||
      static_cast<int>(nb) < n)
    return set_last_error("cuDevSmResourceSplitByCount failed"), SAGE_ERR_INVALID;
  std::unique_ptr<Partition> P(new Partition());
  P->device = device;
  P->total_sms = total;
  for (int i = 0; i < n; ++i) {
    CUdevResourceDesc desc = nullptr;
    Group grp;
    grp.sms = static_cast<int>(res[i].sm.smCount);
    if (g.gen_desc(&desc, &res[i], 1) != CUDA_SUCCESS ||
        g.create(&grp.ctx, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS)
      return set_last_error("green context creation failed"), SAGE_ERR_CUDA;
    P->groups.push_back(grp);
  }
  // the runtime stays on the primary context for everything else
  cudaSetDevice(device);
  *out = P.release();
  return SAGE_OK;
}

sage_status Partition::stream(int i, cudaStream_t* out) {
  if (i < 0 || i >= static_cast<int>(groups.size())) return set_last_error("bad group"), SAGE_ERR_INVALID;
  CUstream s = nullptr;
  if (green().stream_create(&s, groups[i].ctx, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS)
    return set_last_error("cuGreenCtxStreamCreate failed"), SAGE_ERR_CUDA;
  groups[i].streams.push_back(s);
  *out = reinterpret_cast<cudaStream_t>(s);
  return SAGE_OK;
}

}  // namespace sage

struct sage_partition_s {
  sage::Partition* p = nullptr;
  std::vector<cudaStream_t> first;  // one stream per group
};

extern "C" {

sage_status sage_partition_create(int device, int groups, int min_sms, sage_partition* out) {
  if (!out) return sage::set_last_error("null out"), SAGE_ERR_INVALID;
  *out = nullptr;
  sage::Partition* P = nullptr;
  sage_status st = sage::Partition::create(device, groups, min_sms, &P);
  if (st != SAGE_OK) return st;
  std::unique_ptr<sage_partition_s> h(new sage_partition_s());
  h->p = P;
  for (int i = 0; i < groups; ++i) {
    cudaStream_t s = nullptr;
    st = P->stream(i, &s);
    if (st != SAGE_OK) {
      delete P;
      return st;
    }
    h->first.push_back(s);
  }
  *out = h.release();
  return SAGE_OK;
}

int sage_partition_groups(sage_partition p) { return p ? static_cast<int>(p->first.size()) : 0; }

sage_status sage_partition_stream(sage_partition p, int group, void** stream, int* sms) {
  if (!p || group < 0 || group >= static_cast<int>(p->first.size()))
    return sage::set_last_error("bad partition or group"), SAGE_ERR_INVALID;
  if (stream) *stream = p->first[group];
  if (sms) *sms = p->p->groups[group].sms;
  return SAGE_OK;
}

sage_status sage_partition_destroy(sage_partition p) {
  if (!p) return sage::set_last_error("null partition"), SAGE_ERR_INVALID;
  cudaError_t ce = cudaSuccess;
  for (cudaStream_t s : p->first) {
    const cudaError_t c = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = c;
  }
  delete p->p;
  delete p;
  if (ce != cudaSuccess)
    return sage::set_last_error("partition destroyed, but work on its streams had failed on the device"),
           SAGE_ERR_CUDA;
  return SAGE_OK;
}

}  // extern "C"
