// Allocation-free dense solve: dd_dense_solve_noalloc (declared in include/dd.h).
//
// Some callers cannot call cudaMalloc once they are running: an application
// whose own allocator owns every byte of device memory and hands none out
// after start-up, or a latency-bound loop where cudaMalloc's implicit device
// synchronisation and its possible failure are not acceptable.  For them this
// entry point factors and solves one dense complex-symmetric system with the
// same FP64 kernels as dd_factor / dd_solve (one front, 64-wide blocked
// LDL^T, then the tile-parallel substitution) and allocates nothing: every
// byte of scratch lives in the file-scope array below, which each GPU that
// loads this library holds until the process exits.
#include <atomic>
#include <cstring>

#include "../../include/dd.h"
#include "dd_internal.h"

namespace {

constexpr int T = DD_TILE;
constexpr int kMaxN = DD_NOALLOC_MAX_N;          // 512
constexpr int kMaxRhs = DD_NOALLOC_MAX_NRHS;     // 16
constexpr int kMaxTiles = kMaxN / T;             // 8
// tasks of one front with kMaxTiles tiles: diag + panel + update + forward + backward
constexpr int kMaxTasks = kMaxTiles + kMaxTiles * kMaxTiles + kMaxTiles * kMaxTiles * kMaxTiles + 2 * kMaxTiles;

constexpr size_t kFrontBytes = (size_t)kMaxN * kMaxN * sizeof(double2);
constexpr size_t kRhsBytes = (size_t)kMaxN * kMaxRhs * sizeof(double2);
constexpr size_t kTaskBytes = (size_t)kMaxTasks * sizeof(Task);
constexpr size_t kOffFront = 0;
constexpr size_t kOffRhs = kOffFront + kFrontBytes;
constexpr size_t kOffTask = kOffRhs + kRhsBytes;
constexpr size_t kOffDiag = kOffTask + kTaskBytes;                      // int32 diag front ids
constexpr size_t kOffDesc = kOffDiag + 256;                             // FrontDev
constexpr size_t kOffFlags = kOffDesc + 256;                            // 2 x kMaxTiles int32
constexpr size_t kOffStatus = kOffFlags + 256;                          // DevStatus
constexpr size_t kScratchBytes = kOffStatus + 256;

// The scratch.  Host code must not take its address: the name is only a host
// stand-in for the device symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Layout {
  int n, nt, nrhs;
  int n_diag, n_trsm[kMaxTiles], n_upd[kMaxTiles];
  int trsm_off[kMaxTiles], upd_off[kMaxTiles];
  int fwd_off, bwd_off;
};

Layout make_layout(int n, int nrhs) {
  Layout L{};
  L.n = n;
  L.nrhs = nrhs;
  L.nt = (n + T - 1) / T;
  int q = 0;
  for (int k = 0; k < L.nt; ++k) {
    L.trsm_off[k] = q;
    L.n_trsm[k] = L.nt - k - 1;
    q += L.n_trsm[k];
    L.upd_off[k] = q;
    L.n_upd[k] = (L.nt - k - 1) * (L.nt - k) / 2;
    q += L.n_upd[k];
  }
  L.fwd_off = q;
  q += L.nt;
  L.bwd_off = q;
  q += L.nt;
  return L;
}

// One thread writes the front descriptor and the task lists of the single
// front (they depend only on n), and clears the ready flags and the status.
__global__ void k_plan(unsigned char* scratch, int n, int nt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  FrontDev* F = reinterpret_cast<FrontDev*>(scratch + kOffDesc);
  std::memset(F, 0, sizeof(FrontDev));
  F->off = 0;
  F->roff = 0;
  F->ld = nt * T;
  F->ne = n;
  F->ne_pad = nt * T;
  F->nu = 0;
  F->n_int = n;
  F->kind = 0;
  F->sub = 0;
  F->child[0] = F->child[1] = -1;
  F->tile_off = 0;
  Task* t = reinterpret_cast<Task*>(scratch + kOffTask);
  int q = 0;
  for (int k = 0; k < nt; ++k) {
    for (int i = k + 1; i < nt; ++i) t[q++] = Task{0, i, k, 0};
    for (int j = k + 1; j < nt; ++j)
      for (int i = j; i < nt; ++i) t[q++] = Task{0, i, j, 0};
  }
  for (int i = 0; i < nt; ++i) t[q++] = Task{0, i, 0, 0};            // forward: increasing tile
  for (int j = nt - 1; j >= 0; --j) t[q++] = Task{0, j, 0, 0};       // backward: decreasing tile
  reinterpret_cast<int32_t*>(scratch + kOffDiag)[0] = 0;
  int32_t* flags = reinterpret_cast<int32_t*>(scratch + kOffFlags);
  for (int i = 0; i < 2 * kMaxTiles; ++i) flags[i] = 0;
  DevStatus* st = reinterpret_cast<DevStatus*>(scratch + kOffStatus);
  std::memset(st, 0, sizeof(DevStatus));
  st->min_abs_d = 0x7FF0000000000000ull;
}

// front (ld x ld, row-major) <- lower triangle of A (column-major, lda) with
// identity padding; the strictly upper triangle is written with zeros, so no
// value of an earlier call (of another size or ld) survives anywhere in the
// front, although the factor and solve kernels read the lower triangle only
__global__ void k_load_matrix(unsigned char* scratch, int n, int ld, const double2* A, int64_t lda) {
  double2* front = reinterpret_cast<double2*>(scratch + kOffFront);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ld * ld;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    double2 v = make_double2(0.0, 0.0);
    if (c <= r) {
      if (r < n) v = A[r + (int64_t)c * lda];
      else if (r == c) v = make_double2(1.0, 0.0);
    }
    front[e] = v;
  }
}

// rhs block (ld rows x nrhs, row-major) <- b (column-major, ldb), zero padding
__global__ void k_load_rhs(unsigned char* scratch, int n, int ld, int nrhs, const double2* b, int64_t ldb) {
  double2* z = reinterpret_cast<double2*>(scratch + kOffRhs);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ld * nrhs; e += gridDim.x * blockDim.x) {
    const int r = e / nrhs, j = e % nrhs;
    z[e] = r < n ? b[r + (int64_t)j * ldb] : make_double2(0.0, 0.0);
  }
}

__global__ void k_store_x(const unsigned char* scratch, int n, int nrhs, double2* x, int64_t ldx) {
  const double2* z = reinterpret_cast<const double2*>(scratch + kOffRhs);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += gridDim.x * blockDim.x) {
    const int r = e / nrhs, j = e % nrhs;
    x[r + (int64_t)j * ldx] = z[e];
  }
}

// True for memory the kernels of device `dev` may read and write: device
// memory of that same device, or managed memory.  Device memory of another
// GPU is refused (without peer access a kernel touching it would fault).
bool is_device_of(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

constexpr int kMaxDevices = 64;
// Per-device cache of the scratch's device address.  Two host threads making
// their first call at once may both look it up; both store the same value,
// and the atomics keep that a well-defined race.
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on device `dev`, the current device (looked
// up once per device).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return DD_ERR_CUDA;
  unsigned char* a = g_scratch_addr[dev].load(std::memory_order_relaxed);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DD_ERR_CUDA;
    a = static_cast<unsigned char*>(p);
    g_scratch_addr[dev].store(a, std::memory_order_relaxed);
  }
  *out = a;
  return DD_OK;
}

}  // namespace

extern "C" int dd_dense_solve_noalloc(int32_t n, const dd_c128* A, int64_t lda, int32_t nrhs, const dd_c128* b,
                                      int64_t ldb, dd_c128* x, int64_t ldx, void* cuda_stream) {
  if (n < 1 || n > kMaxN || nrhs < 1 || nrhs > kMaxRhs) return DD_ERR_INVALID_ARG;
  if (!A || !b || !x || lda < n || ldb < n || ldx < n) return DD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_CUDA;
  if (!is_device_of(A, dev) || !is_device_of(b, dev) || !is_device_of(x, dev)) return DD_ERR_INVALID_ARG;
  unsigned char* sc = nullptr;
  int st = scratch_address(dev, &sc);
  if (st != DD_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Layout Lo = make_layout(n, nrhs);
  const int ld = Lo.nt * T;
  void* front = sc + kOffFront;
  const FrontDev* fr = reinterpret_cast<const FrontDev*>(sc + kOffDesc);
  const Task* tasks = reinterpret_cast<const Task*>(sc + kOffTask);
  const int32_t* diag_ids = reinterpret_cast<const int32_t*>(sc + kOffDiag);
  int32_t* flags = reinterpret_cast<int32_t*>(sc + kOffFlags);
  DevStatus* dst = reinterpret_cast<DevStatus*>(sc + kOffStatus);

  k_plan<<<1, 32, 0, s>>>(sc, n, Lo.nt);
  k_load_matrix<<<64, 256, 0, s>>>(sc, n, ld, reinterpret_cast<const double2*>(A), lda);
  for (int k = 0; k < Lo.nt; ++k) {
    ddk::launch_diag(0, 0, front, fr, diag_ids, 1, k, dst, s);
    ddk::launch_trsm(0, front, fr, tasks + Lo.trsm_off[k], Lo.n_trsm[k], k, dst, s);
    ddk::launch_update(0, front, fr, tasks + Lo.upd_off[k], Lo.n_upd[k], k, s);
  }
  k_load_rhs<<<16, 256, 0, s>>>(sc, n, ld, nrhs, reinterpret_cast<const double2*>(b), ldb);
  ddk::launch_forward(0, front, sc + kOffRhs, fr, tasks + Lo.fwd_off, Lo.nt, nrhs, flags, 1, dst, s);
  ddk::launch_backward(0, front, sc + kOffRhs, fr, tasks + Lo.bwd_off, Lo.nt, nrhs, nullptr, nullptr, nullptr, 0,
                       flags + kMaxTiles, 1, dst, s);
  k_store_x<<<16, 256, 0, s>>>(sc, n, nrhs, reinterpret_cast<double2*>(x), ldx);
  if (cudaGetLastError() != cudaSuccess) return DD_ERR_CUDA;
  DevStatus host{};
  if (cudaMemcpyAsync(&host, dst, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess) return DD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DD_ERR_CUDA;
  if (host.code == 3) return DD_ERR_SINGULAR_PIVOT;
  if (host.code == 8) return DD_ERR_TIMEOUT;
  return host.code == 0 ? DD_OK : DD_ERR_CUDA;
}
