// noalloc.cu -- k-nearest-neighbour lists without any device allocation.
//
// gmls_knn_noalloc runs the same cell-list build and exact kNN query as
// gmls_cloud + gmls_neighbors, but needs no context and no arena: its scratch
// (bounding box, cell list, cell-ordered coordinates) lives in one
// file-scope static device array.  It exists for callers that cannot allocate
// device memory at the point where they need neighbour lists -- for example a
// solver embedded in a larger simulation code that reserves all device
// memory at start-up and treats any later allocation as an error, because
// cudaMalloc synchronises the device and can fail in the middle of a time
// step.  The caller passes the coordinates and the output buffers; nothing is
// allocated or freed, by this library or by any library it calls.
//
// Limits and sharing:
//  * at most GMLS_NOALLOC_MAX_POINTS particles per call (the array is sized
//    for that; larger clouds are rejected with GMLS_EINVAL);
//  * every GPU that loads the library holds the array until the process ends;
//  * all calls on a device share the one array and it keeps the previous
//    call's contents (the counters that must start at zero are cleared on
//    the caller's stream at the start of every call); calls whose work
//    overlaps on the GPU -- on different streams, or from different host
//    threads -- race on it and must be serialised by the caller;
//  * the first call on a device looks up the array's device address (once
//    per device); make that first call before any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gmls_internal.cuh"

namespace gmls {
void set_global_error(const std::string& msg);
}

namespace {

using namespace gmls;

constexpr int64_t kMaxPoints = GMLS_NOALLOC_MAX_POINTS;
constexpr int64_t kMaxCells = 140000;  // >= cells of any cloud up to kMaxPoints (about n / 2)
constexpr int kMaxPartials = 256;

constexpr size_t up256(size_t v) { return (v + 255) & ~size_t(255); }
// carve of the scratch array (byte offsets)
constexpr size_t kOffGrid = 0;
constexpr size_t kOffPart = kOffGrid + up256(sizeof(GridParams));
constexpr size_t kOffCellOf = kOffPart + up256(sizeof(double) * 6 * kMaxPartials);
constexpr size_t kOffCounts = kOffCellOf + up256(sizeof(int32_t) * kMaxPoints);
constexpr size_t kOffFill = kOffCounts + up256(sizeof(int32_t) * kMaxCells);
constexpr size_t kOffStart = kOffFill + up256(sizeof(int32_t) * kMaxCells);
constexpr size_t kOffScan = kOffStart + up256(sizeof(int32_t) * (kMaxCells + 1));
constexpr size_t kOffSorted = kOffScan + up256(sizeof(int32_t) * (kMaxCells / 2048 + 4));
constexpr size_t kOffXs = kOffSorted + up256(sizeof(int32_t) * kMaxPoints);
constexpr size_t kOffXsf = kOffXs + up256(sizeof(double) * 3 * kMaxPoints);
constexpr size_t kScratchBytes = kOffXsf + up256(sizeof(float) * 3 * kMaxPoints);  // about 13.7 MB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

gmls_status err(gmls_status code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

// device (or managed) memory of device dev: the kernels run on the current
// device and must not reach into a peer's memory
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" gmls_status gmls_knn_noalloc(int dim, int64_t n, const double* xyz, int32_t k, double eps_factor,
                                        int32_t* out_idx, double* out_eps, uint8_t* out_status, void* cuda_stream) {
  if ((dim != 2 && dim != 3) || n < 1 || k < 1 || k > kMaxK || k > n || !(eps_factor > 0.0))
    return err(GMLS_EINVAL, "gmls_knn_noalloc: need dim in {2,3}, 1 <= k <= min(n, 1024), eps_factor > 0");
  if (n > kMaxPoints)
    return err(GMLS_EINVAL, "gmls_knn_noalloc: at most " + std::to_string(kMaxPoints) +
                                " particles (the static scratch array is sized for that); got " + std::to_string(n));
  if (!xyz || !out_idx || !out_eps || !out_status)
    return err(GMLS_EINVAL, "gmls_knn_noalloc: NULL pointer");
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return err(GMLS_ECUDA, "gmls_knn_noalloc: no current CUDA device");
  }
  if (!on_device(xyz, cur) || !on_device(out_idx, cur) || !on_device(out_eps, cur) || !on_device(out_status, cur))
    return err(GMLS_EINVAL, "gmls_knn_noalloc: coordinates and outputs must be device memory of the current device (" +
                                std::to_string(cur) + ")");
  int32_t nc_axis[3] = {1, 1, 1};
  const double per_axis = std::pow(std::max(1.0, n / 2.0), 1.0 / dim);
  int64_t ncell = 1;
  for (int a = 0; a < dim; ++a) {
    nc_axis[a] = std::max(1, (int)std::ceil(per_axis));
    ncell *= nc_axis[a];
  }
  if (ncell > kMaxCells) return err(GMLS_EINVAL, "gmls_knn_noalloc: cell grid exceeds the scratch array");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(GMLS_ECUDA, std::string("gmls_knn_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {  // once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess)
        return err(GMLS_ECUDA, std::string("gmls_knn_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_addr[dev];
  }
  GridParams* grid = reinterpret_cast<GridParams*>(base + kOffGrid);
  double* part = reinterpret_cast<double*>(base + kOffPart);
  int32_t* cell_of = reinterpret_cast<int32_t*>(base + kOffCellOf);
  int32_t* counts = reinterpret_cast<int32_t*>(base + kOffCounts);
  int32_t* fill = reinterpret_cast<int32_t*>(base + kOffFill);
  int32_t* cell_start = reinterpret_cast<int32_t*>(base + kOffStart);
  int32_t* scan_tmp = reinterpret_cast<int32_t*>(base + kOffScan);
  int32_t* sorted = reinterpret_cast<int32_t*>(base + kOffSorted);
  double* xs = reinterpret_cast<double*>(base + kOffXs);
  float* xsf = reinterpret_cast<float*>(base + kOffXsf);
  const int64_t scan_elems = kMaxCells / 2048 + 4;
  const int n_part = (int)std::min<int64_t>(kMaxPartials, (n + 255) / 256);

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int64_t launches = 0;
  Launch L{s, &launches};
  // the previous call's counters are still in the array: clear them
  if ((e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * ncell, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * ncell, s)) != cudaSuccess ||
      (e = launch_bbox_and_grid(L, dim, n, xyz, nc_axis, grid, part, n_part)) != cudaSuccess ||
      (e = launch_cell_count(L, dim, n, xyz, grid, cell_of, counts)) != cudaSuccess ||
      (e = launch_scan_i32(L, counts, cell_start, ncell, scan_tmp, scan_elems)) != cudaSuccess ||
      (e = launch_cell_scatter(L, dim, n, xyz, grid, cell_of, cell_start, fill, sorted, xs, xsf)) != cudaSuccess)
    return err(GMLS_ECUDA, std::string("gmls_knn_noalloc: cell list: ") + cudaGetErrorString(e));
  NbrQuery q;
  std::memset(&q, 0, sizeof(q));
  q.cloud = CloudDev{dim, n, xyz, xs, sorted, cell_start, grid, ncell, xsf};
  q.n_tgt = n;
  q.tgt = nullptr;
  q.halfspace = nullptr;
  q.mode = GMLS_NBR_KNN;
  q.k = k;
  q.cap = k;
  q.eps_factor = eps_factor;
  q.out_idx = out_idx;
  q.out_cnt = nullptr;
  q.out_eps = out_eps;
  q.out_status = out_status;
  if ((e = launch_nbr_query(L, q)) != cudaSuccess)
    return err(GMLS_ECUDA, std::string("gmls_knn_noalloc: query: ") + cudaGetErrorString(e));
  return GMLS_OK;
}
