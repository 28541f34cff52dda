// Cross-process sharing of a function's read-only copy (the paper's memory daemon
// as a separate process, Sec. 4.1 / Sec. 5.1, sharing of read-only data between
// invocations, Sec. 6.2).
//
// Owner: a pool created exportable allocates each read-only item as CUDA VMM
// physical memory with a POSIX file-descriptor handle.  sage_share_start listens
// on a UNIX SOCK_SEQPACKET socket; each connection is one attach:
//
//   function process                          owner
//   ATTACH {key, shape signature}  ------->   sage_prepare (first attach stages)
//                                  <-------   GRANT {status, sizes, GPU uuid} + 2 fds
//                                  <-------   READY {status}   (staging finished)
//   close (release / exit)         ------->   sage_release
//
// The function process sends ATTACH before it creates its context, so the owner's
// staging overlaps the context creation; it maps the two blocks, builds its own
// workspaces and returns a handle whose readiness gate opens on READY.
#include <errno.h>
#include <string.h>
#include <sys/socket.h>
#include <sys/time.h>
#include <sys/un.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sage.h"
#include "kernels.h"

namespace sage {
namespace {

// ---------------------------------------------------------------- VMM entry points

struct Vmm {
  decltype(&cuMemCreate) create = nullptr;
  decltype(&cuMemRelease) release = nullptr;
  decltype(&cuMemAddressReserve) reserve = nullptr;
  decltype(&cuMemAddressFree) addr_free = nullptr;
  decltype(&cuMemMap) map = nullptr;
  decltype(&cuMemUnmap) unmap = nullptr;
  decltype(&cuMemSetAccess) set_access = nullptr;
  decltype(&cuMemGetAllocationGranularity) granularity = nullptr;
  decltype(&cuMemExportToShareableHandle) export_handle = nullptr;
  decltype(&cuMemImportFromShareableHandle) import_handle = nullptr;
  bool ok = false;
};

template <class F>
void entry(const char* name, F* out) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    *out = reinterpret_cast<F>(p);
}

const Vmm& vmm() {
  static Vmm v;
  static std::once_flag once;
  std::call_once(once, [] {
    entry("cuMemCreate", &v.create);
    entry("cuMemRelease", &v.release);
    entry("cuMemAddressReserve", &v.reserve);
    entry("cuMemAddressFree", &v.addr_free);
    entry("cuMemMap", &v.map);
    entry("cuMemUnmap", &v.unmap);
    entry("cuMemSetAccess", &v.set_access);
    entry("cuMemGetAllocationGranularity", &v.granularity);
    entry("cuMemExportToShareableHandle", &v.export_handle);
    entry("cuMemImportFromShareableHandle", &v.import_handle);
    v.ok = v.create && v.release && v.reserve && v.addr_free && v.map && v.unmap && v.set_access &&
           v.granularity && v.export_handle && v.import_handle;
  });
  return v;
}

CUmemAllocationProp device_prop(int device) {
  CUmemAllocationProp p;
  memset(&p, 0, sizeof(p));
  p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  p.location.id = device;
  p.requestedHandleTypes = CU_MEM_HANDLE_TYPE_POSIX_FILE_DESCRIPTOR;
  return p;
}

// Reserve an address range for `h` (size bytes), map it and allow read-write
// access from `device`.  Releases nothing on failure (the caller owns h).
bool map_handle(int device, CUmemGenericAllocationHandle h, size_t size, size_t align, void** va) {
  const Vmm& v = vmm();
  CUdeviceptr d = 0;
  if (v.reserve(&d, size, align, 0, 0) != CUDA_SUCCESS) return false;
  if (v.map(d, size, 0, h, 0) != CUDA_SUCCESS) {
    v.addr_free(d, size);
    return false;
  }
  CUmemAccessDesc a;
  memset(&a, 0, sizeof(a));
  a.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  a.location.id = device;
  a.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  if (v.set_access(d, size, &a, 1) != CUDA_SUCCESS) {
    v.unmap(d, size);
    v.addr_free(d, size);
    return false;
  }
  *va = reinterpret_cast<void*>(d);
  return true;
}

size_t granularity(int device) {
  const CUmemAllocationProp p = device_prop(device);
  size_t g = 0;
  if (vmm().granularity(&g, &p, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || g == 0) g = size_t(2) << 20;
  return g;
}

// Import an exported block (takes the descriptor) and map it here.
bool vmm_import(int device, int fd, size_t size, VmmBlock* out) {
  const Vmm& v = vmm();
  CUmemGenericAllocationHandle h = 0;
  const CUresult r = v.import_handle(&h, reinterpret_cast<void*>(static_cast<intptr_t>(fd)),
                                     CU_MEM_HANDLE_TYPE_POSIX_FILE_DESCRIPTOR);
  close(fd);
  if (r != CUDA_SUCCESS) return false;
  void* va = nullptr;
  if (!map_handle(device, h, size, granularity(device), &va)) {
    v.release(h);
    return false;
  }
  out->handle = h;
  out->va = va;
  out->size = size;
  return true;
}

// ---------------------------------------------------------------- protocol

enum : int32_t { kAttach = 1, kGrant = 2, kReady = 3 };
constexpr uint32_t kMagic = 0x45474153u;  // "SAGE"

struct Msg {
  uint32_t magic = kMagic;
  int32_t type = 0;
  int32_t status = 0;
  int32_t nfd = 0;
  uint64_t tables_bytes = 0, weights_bytes = 0;
  uint64_t tables_map = 0, weights_map = 0;  // mapped sizes of the exported blocks
  uint8_t uuid[16] = {};
  char key[256] = {};
  char sig[4096] = {};
};

bool send_msg(int fd, const Msg& m, const int* fds, int nfds) {
  iovec io{const_cast<Msg*>(&m), sizeof(Msg)};
  msghdr h;
  memset(&h, 0, sizeof(h));
  h.msg_iov = &io;
  h.msg_iovlen = 1;
  alignas(cmsghdr) char ctl[CMSG_SPACE(2 * sizeof(int))];
  if (nfds > 0) {
    memset(ctl, 0, sizeof(ctl));
    h.msg_control = ctl;
    h.msg_controllen = CMSG_SPACE(nfds * sizeof(int));
    cmsghdr* c = CMSG_FIRSTHDR(&h);
    c->cmsg_level = SOL_SOCKET;
    c->cmsg_type = SCM_RIGHTS;
    c->cmsg_len = CMSG_LEN(nfds * sizeof(int));
    memcpy(CMSG_DATA(c), fds, nfds * sizeof(int));
  }
  for (;;) {
    const ssize_t n = sendmsg(fd, &h, MSG_NOSIGNAL);
    if (n == static_cast<ssize_t>(sizeof(Msg))) return true;
    if (n < 0 && errno == EINTR) continue;
    return false;
  }
}

// 1: a whole message (fds received into fds[0..*nfds)); 0: the peer closed;
// -1: error; -2: receive timeout.
int recv_msg(int fd, Msg* m, int* fds, int* nfds, int maxfds) {
  iovec io{m, sizeof(Msg)};
  msghdr h;
  memset(&h, 0, sizeof(h));
  h.msg_iov = &io;
  h.msg_iovlen = 1;
  alignas(cmsghdr) char ctl[CMSG_SPACE(2 * sizeof(int))];
  h.msg_control = ctl;
  h.msg_controllen = sizeof(ctl);
  if (nfds) *nfds = 0;
  ssize_t n;
  do {
    n = recvmsg(fd, &h, MSG_CMSG_CLOEXEC);
  } while (n < 0 && errno == EINTR);
  if (n == 0) return 0;
  if (n < 0) return (errno == EAGAIN || errno == EWOULDBLOCK) ? -2 : -1;
  int got = 0;
  for (cmsghdr* c = CMSG_FIRSTHDR(&h); c; c = CMSG_NXTHDR(&h, c)) {
    if (c->cmsg_level != SOL_SOCKET || c->cmsg_type != SCM_RIGHTS) continue;
    const int k = static_cast<int>((c->cmsg_len - CMSG_LEN(0)) / sizeof(int));
    int tmp[4];
    memcpy(tmp, CMSG_DATA(c), std::min(k, 4) * sizeof(int));
    for (int i = 0; i < k && i < 4; ++i) {
      if (fds && got < maxfds) fds[got++] = tmp[i];
      else close(tmp[i]);
    }
  }
  if (nfds) *nfds = got;
  const bool whole = n == static_cast<ssize_t>(sizeof(Msg)) && !(h.msg_flags & MSG_TRUNC) && m->magic == kMagic;
  if (!whole) {
    for (int i = 0; i < got; ++i) close(fds[i]);
    if (nfds) *nfds = 0;
    return -1;
  }
  return 1;
}

bool fill_addr(const char* path, sockaddr_un* a) {
  if (!path || strlen(path) == 0 || strlen(path) >= sizeof(a->sun_path)) return false;
  memset(a, 0, sizeof(*a));
  a->sun_family = AF_UNIX;
  strncpy(a->sun_path, path, sizeof(a->sun_path) - 1);
  return true;
}

void set_rcv_timeout(int fd, double seconds) {
  timeval tv;
  tv.tv_sec = static_cast<time_t>(seconds);
  tv.tv_usec = static_cast<suseconds_t>((seconds - static_cast<double>(tv.tv_sec)) * 1e6);
  setsockopt(fd, SOL_SOCKET, SO_RCVTIMEO, &tv, sizeof(tv));
}

bool device_uuid(int device, uint8_t out[16]) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  memcpy(out, p.uuid.bytes, 16);
  return true;
}

// A descriptor with its own copies of the key, rows and layer sizes.
struct OwnedDesc {
  std::string key;
  std::vector<int64_t> rows;
  std::vector<int> bot, top;
  sage_fn_desc d{};
  std::string sig;
  explicit OwnedDesc(const sage_fn_desc* s)
      : key(s->fn_key), rows(s->rows, s->rows + s->num_tables), bot(s->bot_dims, s->bot_dims + s->n_bot),
        top(s->top_dims, s->top_dims + s->n_top), d(*s) {
    d.fn_key = key.c_str();
    d.rows = rows.data();
    d.bot_dims = bot.data();
    d.top_dims = top.data();
    d.tables.key = key.c_str();
    d.weights.key = key.c_str();
    sig = shape_signature(&d);
  }
};

// The function process's side of one attach: the mapped blocks and the socket
// on which READY arrives (closing it returns the owner's reference).
struct SocketImport : ImportedData {
  int fd = -1;
  VmmBlock t, w;
  bool wait_ready() override {
    Msg m;
    return recv_msg(fd, &m, nullptr, nullptr, 0) == 1 && m.type == kReady && m.status == SAGE_OK;
  }
  void interrupt() override { shutdown(fd, SHUT_RDWR); }
  ~SocketImport() override {
    vmm_free(t);
    vmm_free(w);
    if (fd >= 0) close(fd);
  }
};

}  // namespace

bool vmm_alloc(int device, size_t bytes, VmmBlock* out) {
  const Vmm& v = vmm();
  if (!v.ok) {
    set_last_error("CUDA virtual memory management entry points unavailable");
    return false;
  }
  const CUmemAllocationProp p = device_prop(device);
  const size_t g = granularity(device);
  const size_t size = (bytes + g - 1) / g * g;
  CUmemGenericAllocationHandle h = 0;
  if (v.create(&h, size, &p, 0) != CUDA_SUCCESS) {
    set_last_error("cuMemCreate of exportable device memory failed");
    return false;
  }
  void* va = nullptr;
  if (!map_handle(device, h, size, g, &va)) {
    v.release(h);
    set_last_error("mapping exportable device memory failed");
    return false;
  }
  out->handle = h;
  out->va = va;
  out->size = size;
  return true;
}

void vmm_free(VmmBlock& b) {
  if (!b.va) return;
  const Vmm& v = vmm();
  const CUdeviceptr d = reinterpret_cast<CUdeviceptr>(b.va);
  v.unmap(d, b.size);
  v.addr_free(d, b.size);
  v.release(b.handle);
  b = VmmBlock();
}

}  // namespace sage

// ---------------------------------------------------------------- owner

using sage::Msg;

struct ShareConn {
  int fd = -1;
  std::thread th;
  std::atomic<bool> done{false};
};

struct sage_share_s {
  sage_pool pool = nullptr;
  int device = 0;
  uint8_t uuid[16] = {};
  std::string path;
  int lfd = -1;
  std::thread acceptor;
  std::atomic<bool> stop{false};
  std::mutex mu;
  std::unordered_map<std::string, std::unique_ptr<sage::OwnedDesc>> reg;
  std::list<std::unique_ptr<ShareConn>> conns;
  sage_share_stats st{};

  void serve(ShareConn* c);
  void grant_fail(int fd, sage_status s) {
    Msg r;
    r.type = sage::kGrant;
    r.status = s;
    sage::send_msg(fd, r, nullptr, 0);
    std::lock_guard<std::mutex> g(mu);
    st.rejects++;
  }
};

void sage_share_s::serve(ShareConn* c) {
  const int fd = c->fd;
  Msg m;
  const int r = sage::recv_msg(fd, &m, nullptr, nullptr, 0);
  sage::OwnedDesc* od = nullptr;
  if (r == 1 && m.type == sage::kAttach) {
    m.key[sizeof(m.key) - 1] = 0;
    m.sig[sizeof(m.sig) - 1] = 0;
    std::lock_guard<std::mutex> g(mu);
    st.connections++;
    auto it = reg.find(m.key);
    if (it != reg.end() && it->second->sig == m.sig) od = it->second.get();
  }
  sage_fn f = nullptr;
  if (r == 1 && m.type == sage::kAttach) {
    if (!od) {
      grant_fail(fd, SAGE_ERR_INVALID);
    } else {
      cudaSetDevice(device);
      sage_status s = sage_prepare(pool, &od->d, &f);
      sage::VmmBlock t, w;
      if (s == SAGE_OK) s = sage::fn_export(f, &t, &w);
      int fds[2] = {-1, -1};
      if (s == SAGE_OK) {
        const sage::Vmm& v = sage::vmm();
        if (v.export_handle(&fds[0], t.handle, CU_MEM_HANDLE_TYPE_POSIX_FILE_DESCRIPTOR, 0) != CUDA_SUCCESS ||
            v.export_handle(&fds[1], w.handle, CU_MEM_HANDLE_TYPE_POSIX_FILE_DESCRIPTOR, 0) != CUDA_SUCCESS)
          s = SAGE_ERR_CUDA;
      }
      if (s != SAGE_OK) {
        for (int x : fds)
          if (x >= 0) close(x);
        if (f) sage_release(f);
        f = nullptr;
        grant_fail(fd, s);
      } else {
        Msg g;
        g.type = sage::kGrant;
        g.status = SAGE_OK;
        g.nfd = 2;
        g.tables_bytes = od->d.tables.bytes;
        g.weights_bytes = od->d.weights.bytes;
        g.tables_map = t.size;
        g.weights_map = w.size;
        memcpy(g.uuid, uuid, 16);
        const bool sent = sage::send_msg(fd, g, fds, 2);
        close(fds[0]);
        close(fds[1]);
        {
          std::lock_guard<std::mutex> lk(mu);
          if (sent) st.grants++, st.active++;
        }
        if (!sent) {
          sage_release(f);
          f = nullptr;
        }
      }
    }
  }
  if (f) {
    // READY once staging has finished (or failed); stop interrupts the wait
    sage_status s;
    do {
      s = sage_wait(f, 100000);
    } while (s == SAGE_ERR_TIMEOUT && !stop.load());
    Msg rd;
    rd.type = sage::kReady;
    rd.status = s == SAGE_ERR_TIMEOUT ? SAGE_ERR_STAGING : s;
    if (sage::send_msg(fd, rd, nullptr, 0)) {
      std::lock_guard<std::mutex> g(mu);
      st.ready++;
    }
    // hold the reference until the function process closes (or the owner stops)
    char buf[64];
    while (recv(fd, buf, sizeof(buf), 0) > 0) {
    }
    sage_release(f);
    std::lock_guard<std::mutex> g(mu);
    st.releases++;
    st.active--;
  }
  c->done.store(true);  // the socket is closed by whoever joins this thread
}

extern "C" {

sage_status sage_share_start(sage_pool pool, const char* socket_path, sage_share* out) {
  if (!pool || !out) return sage::set_last_error("null pool or out"), SAGE_ERR_INVALID;
  *out = nullptr;
  sockaddr_un a;
  if (!sage::fill_addr(socket_path, &a)) return sage::set_last_error("bad socket path"), SAGE_ERR_INVALID;
  if (!sage::pool_exportable(pool))
    return sage::set_last_error("the pool was not created exportable"), SAGE_ERR_INVALID;
  std::unique_ptr<sage_share_s> S(new sage_share_s());
  S->pool = pool;
  S->path = socket_path;
  if (cudaGetDevice(&S->device) != cudaSuccess || !sage::device_uuid(S->device, S->uuid))
    return sage::set_last_error("no CUDA device"), SAGE_ERR_CUDA;
  if (!sage::vmm().ok) return sage::set_last_error("CUDA VMM entry points unavailable"), SAGE_ERR_CUDA;
  unlink(socket_path);
  S->lfd = socket(AF_UNIX, SOCK_SEQPACKET | SOCK_CLOEXEC, 0);
  if (S->lfd < 0) return sage::set_last_error("socket() failed"), SAGE_ERR_CUDA;
  if (bind(S->lfd, reinterpret_cast<sockaddr*>(&a), sizeof(a)) != 0 || listen(S->lfd, 64) != 0) {
    close(S->lfd);
    return sage::set_last_error("cannot listen on the socket path"), SAGE_ERR_CUDA;
  }
  sage_share_s* raw = S.get();
  S->acceptor = std::thread([raw] {
    for (;;) {
      const int fd = accept4(raw->lfd, nullptr, nullptr, SOCK_CLOEXEC);
      if (fd < 0) {
        if (errno == EINTR || errno == ECONNABORTED) continue;
        return;  // the listening socket was shut down
      }
      std::lock_guard<std::mutex> g(raw->mu);
      if (raw->stop.load()) {
        close(fd);
        return;
      }
      // reap finished connections
      for (auto it = raw->conns.begin(); it != raw->conns.end();) {
        if ((*it)->done.load()) {
          (*it)->th.join();
          close((*it)->fd);
          it = raw->conns.erase(it);
        } else {
          ++it;
        }
      }
      raw->conns.emplace_back(new ShareConn());
      ShareConn* c = raw->conns.back().get();
      c->fd = fd;
      c->th = std::thread([raw, c] { raw->serve(c); });
    }
  });
  *out = S.release();
  return SAGE_OK;
}

sage_status sage_share_register(sage_share S, const sage_fn_desc* d) {
  if (!S || !d) return sage::set_last_error("null share or descriptor"), SAGE_ERR_INVALID;
  sage_status s = sage::check_shape(d);
  if (s != SAGE_OK) return s;
  if ((!d->tables.host_src) == (!d->tables.fill) || (!d->weights.host_src) == (!d->weights.fill))
    return sage::set_last_error("each data item needs exactly one of host_src or fill"), SAGE_ERR_INVALID;
  std::unique_ptr<sage::OwnedDesc> od(new sage::OwnedDesc(d));
  std::lock_guard<std::mutex> g(S->mu);
  S->reg[od->key] = std::move(od);
  return SAGE_OK;
}

sage_status sage_share_stats_get(sage_share S, sage_share_stats* out) {
  if (!S || !out) return sage::set_last_error("null share or out"), SAGE_ERR_INVALID;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->st;
  return SAGE_OK;
}

sage_status sage_share_stop(sage_share S) {
  if (!S) return sage::set_last_error("null share"), SAGE_ERR_INVALID;
  S->stop.store(true);
  shutdown(S->lfd, SHUT_RDWR);
  if (S->acceptor.joinable()) S->acceptor.join();
  close(S->lfd);
  std::list<std::unique_ptr<ShareConn>> conns;
  {
    std::lock_guard<std::mutex> g(S->mu);
    conns.swap(S->conns);
  }
  for (auto& c : conns) shutdown(c->fd, SHUT_RDWR);
  for (auto& c : conns) {
    if (c->th.joinable()) c->th.join();
    close(c->fd);
  }
  unlink(S->path.c_str());
  delete S;
  return SAGE_OK;
}

// ---------------------------------------------------------------- function process

struct sage_ticket_s {
  int fd = -1;
  std::unique_ptr<sage::OwnedDesc> shape;
};

sage_status sage_attach_begin(const char* socket_path, const sage_fn_desc* shape, sage_ticket* out) {
  if (!out) return sage::set_last_error("null out"), SAGE_ERR_INVALID;
  *out = nullptr;
  sage_status s = sage::check_shape(shape);
  if (s != SAGE_OK) return s;
  sockaddr_un a;
  if (!sage::fill_addr(socket_path, &a)) return sage::set_last_error("bad socket path"), SAGE_ERR_INVALID;
  std::unique_ptr<sage_ticket_s> t(new sage_ticket_s());
  t->shape.reset(new sage::OwnedDesc(shape));
  if (t->shape->sig.size() >= sizeof(Msg::sig)) return sage::set_last_error("shape too large"), SAGE_ERR_INVALID;
  t->fd = socket(AF_UNIX, SOCK_SEQPACKET | SOCK_CLOEXEC, 0);
  if (t->fd < 0) return sage::set_last_error("socket() failed"), SAGE_ERR_INVALID;
  if (connect(t->fd, reinterpret_cast<sockaddr*>(&a), sizeof(a)) != 0) {
    close(t->fd);
    return sage::set_last_error("no owner listens on the socket path"), SAGE_ERR_INVALID;
  }
  Msg m;
  m.type = sage::kAttach;
  strncpy(m.key, t->shape->key.c_str(), sizeof(m.key) - 1);
  strncpy(m.sig, t->shape->sig.c_str(), sizeof(m.sig) - 1);
  if (!sage::send_msg(t->fd, m, nullptr, 0)) {
    close(t->fd);
    return sage::set_last_error("sending the attach request failed"), SAGE_ERR_INVALID;
  }
  *out = t.release();
  return SAGE_OK;
}

sage_status sage_attach_cancel(sage_ticket ticket) {
  if (!ticket) return sage::set_last_error("null ticket"), SAGE_ERR_INVALID;
  if (ticket->fd >= 0) close(ticket->fd);
  delete ticket;
  return SAGE_OK;
}

sage_status sage_attach_end(sage_pool pool, sage_ticket ticket, sage_fn* out) {
  std::unique_ptr<sage_ticket_s> t(ticket);
  if (!pool || !t || !out) {
    if (t && t->fd >= 0) close(t->fd);
    return sage::set_last_error("null pool, ticket or out"), SAGE_ERR_INVALID;
  }
  *out = nullptr;
  std::unique_ptr<sage::SocketImport> imp(new sage::SocketImport());
  imp->fd = t->fd;  // closed with imp from here on
  t->fd = -1;
  sage::set_rcv_timeout(imp->fd, 60.0);
  Msg g;
  int fds[2] = {-1, -1}, nfd = 0;
  const int r = sage::recv_msg(imp->fd, &g, fds, &nfd, 2);
  if (r == -2) return sage::set_last_error("the owner did not answer within 60 s"), SAGE_ERR_TIMEOUT;
  if (r != 1 || g.type != sage::kGrant) {
    for (int i = 0; i < nfd; ++i) close(fds[i]);
    return sage::set_last_error("the owner closed the attach"), SAGE_ERR_INVALID;
  }
  if (g.status != SAGE_OK) {
    for (int i = 0; i < nfd; ++i) close(fds[i]);
    sage::set_last_error("the owner refused the attach (unknown key, other shape, or its prepare failed)");
    return static_cast<sage_status>(g.status);
  }
  if (nfd != 2 || g.tables_bytes != t->shape->d.tables.bytes || g.weights_bytes != t->shape->d.weights.bytes ||
      g.tables_map < g.tables_bytes || g.weights_map < g.weights_bytes) {
    for (int i = 0; i < nfd; ++i) close(fds[i]);
    return sage::set_last_error("malformed grant"), SAGE_ERR_INVALID;
  }
  const int dev = sage::pool_device(pool);
  uint8_t mine[16];
  if (cudaSetDevice(dev) != cudaSuccess || !sage::device_uuid(dev, mine) || memcmp(mine, g.uuid, 16) != 0) {
    close(fds[0]);
    close(fds[1]);
    return sage::set_last_error("the owner's copy lives on another GPU"), SAGE_ERR_INVALID;
  }
  const bool mt = sage::vmm_import(dev, fds[0], g.tables_map, &imp->t);
  const bool mw = sage::vmm_import(dev, fds[1], g.weights_map, &imp->w);
  if (!mt || !mw) return sage::set_last_error("mapping the owner's copy failed"), SAGE_ERR_CUDA;
  sage::set_rcv_timeout(imp->fd, 0.0);  // READY may take as long as the staging
  imp->tables = static_cast<char*>(imp->t.va);
  imp->weights = static_cast<char*>(imp->w.va);
  return sage::prepare_imported(pool, &t->shape->d, imp.release(), out);
}

}  // extern "C"
