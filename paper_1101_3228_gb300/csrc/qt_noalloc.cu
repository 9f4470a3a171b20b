// qt_noalloc.cu -- qt_counts_from_samples_noalloc: the counting step of
// Algorithm III on caller-supplied samples, for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host application whose own allocator
// has reserved the device memory up front, a plug-in that is not allowed to own
// device memory, or a latency-bound loop in which the implicit synchronisation
// of cudaMalloc/cudaFree is not acceptable.  This entry point needs no context
// and no allocation: the caller passes the grids, the samples and the output
// buffers, and every scratch byte the kernels need (status word and work-queue
// counter, the layer and grid descriptors, a contiguous copy of both grids and
// their screened FP32 records) lives in the file-scope array below, one copy
// per device that loads the library, held until the process exits.
//
// Limits: d <= 16 and NA + NB <= QT_NOALLOC_MAX_POINTS (4096) points; the
// screened records of both grids must also fit the shared memory of one CTA
// (the same rule as qt_counts_from_samples).  Larger inputs are rejected with
// QT_EINVAL before anything is enqueued.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/qt.h"
#include "qt_internal.h"
#include "qt_launch.h"

namespace qt {
__global__ void prep_records_kernel(const double*, GridInfo*, int, int, int, int, long long, float*, double*);
}

using namespace qt;

namespace {

constexpr long long kMaxPoints = QT_NOALLOC_MAX_POINTS;
constexpr long long kMaxRecs = kMaxPoints + 2 * kChunk;     // both grids padded to whole chunks
constexpr long long kRecFloatsMax = 20;                     // d = 16: [cc, 16 coordinates, 3 zeros]
constexpr size_t kOffStatus = 0;
constexpr size_t kOffLayer = 256;
constexpr size_t kOffGrids = 512;
constexpr size_t kOffG64 = 1024;
constexpr size_t kOffRec = kOffG64 + (size_t)kMaxPoints * kDMax * sizeof(double);
constexpr size_t kScratchBytes = kOffRec + (size_t)kMaxRecs * kRecFloatsMax * sizeof(float);

static_assert(sizeof(DevStatus) <= 256 && sizeof(LayerDesc) <= 256 && 2 * sizeof(GridInfo) <= 512, "layout");

// The scratch of every call on this device.  In host code this name is only a
// stand-in for the symbol, never a device address: the address comes from
// cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char qt_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// What a call needs to know about its device, looked up once per device.
struct DeviceSetup {
    void* scratch = nullptr;   // device address of qt_noalloc_scratch on this device
    int num_sms = 0;           // multiprocessors (grid size of the persistent kernel)
    int smem_optin = 0;        // opt-in shared memory per block (the resident-grid budget)
};
std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the device address of the array
// and the two device attributes the plan needs (cudaDeviceGetAttribute, so that
// later calls query nothing).
cudaError_t device_setup(int dev, DeviceSetup* out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.scratch) {
        DeviceSetup n;
        cudaError_t e = cudaDeviceGetAttribute(&n.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&n.scratch, qt_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        s = n;
    }
    *out = s;
    return cudaSuccess;
}

int dim_class(int d)
{
    static const int dms[] = {1, 2, 3, 4, 6, 8, 10, 12, 16};
    for (int v : dms)
        if (v >= d) return v;
    return 0;
}

long long up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace

extern "C" qt_status qt_counts_from_samples_noalloc(int32_t d, const double* gA, int64_t NA, const double* gB,
                                                    int64_t NB, const double* X, const double* Y, int64_t M,
                                                    int32_t counts_type, void* counts, int32_t* ii, int32_t* jj,
                                                    void* stream)
{
    if (d < 1 || d > kDMax) return QT_EINVAL;
    if (!gA || !gB || !X || !Y || !counts) return QT_EINVAL;
    if (NA < 1 || NB < 1 || NA + NB > kMaxPoints) return QT_EINVAL;
    if (M < 1 || M > 0xFFFFFFFFll) return QT_EINVAL;
    if ((ii == nullptr) != (jj == nullptr)) return QT_EINVAL;
    if (counts_type != QT_COUNTS_I64 && counts_type != QT_COUNTS_U32) return QT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QT_ECUDA;
    DeviceSetup ds;
    if (device_setup(dev, &ds) != cudaSuccess) return QT_ECUDA;
    unsigned char* base = static_cast<unsigned char*>(ds.scratch);

    // plan: FP32 screen with FP64 recheck, both grids resident in shared memory
    const int dm = dim_class(d);
    const int rec_floats = 4 * ((dm + 1 + 3) / 4);
    const int S = dm <= 2 ? 8 : (dm <= 4 ? 4 : 2);
    const int block = 256;
    const long long NApad = up(NA, kChunk), NBpad = up(NB, kChunk);
    const size_t grid_bytes = (size_t)up((NApad + NBpad) * rec_floats * 4, 128);
    const size_t budget = ds.smem_optin > 24 * 1024 ? (size_t)ds.smem_optin - 24 * 1024 : 0;
    if (grid_bytes > budget || !forward_variant_exists(kF32Recheck, dm, S, false)) return QT_EINVAL;

    DevStatus* dstatus = reinterpret_cast<DevStatus*>(base + kOffStatus);
    LayerDesc* dlayer = reinterpret_cast<LayerDesc*>(base + kOffLayer);
    GridInfo* dgrids = reinterpret_cast<GridInfo*>(base + kOffGrids);
    double* dg64 = reinterpret_cast<double*>(base + kOffG64);
    float* drec = reinterpret_cast<float*>(base + kOffRec);

    // descriptors (host stack, copied into the scratch)
    GridInfo G[2];
    memset(G, 0, sizeof G);
    G[0].N = (int)NA;
    G[0].Npad = (int)NApad;
    G[0].goff = 0;
    G[0].roff = 0;
    G[1].N = (int)NB;
    G[1].Npad = (int)NBpad;
    G[1].goff = NA;
    G[1].roff = NApad;
    LayerDesc L;
    memset(&L, 0, sizeof L);
    const int tile = block * S;
    L.NA = (int)NA;
    L.NB = (int)NB;
    L.NApad = (int)NApad;
    L.NBpad = (int)NBpad;
    L.gridA = 0;
    L.gridB = 1;
    L.goffA = 0;
    L.goffB = NA;
    L.roffA = 0;
    L.roffB = NApad;
    L.coff = 0;
    L.item_begin = 0;
    L.items = (int)((M + tile - 1) / tile);
    L.hist_smem = 0;

    const size_t csize = counts_type == QT_COUNTS_U32 ? 4 : 8;
    // everything that must start at zero is cleared: status word, queue, counts;
    // the grid tables carry R = 0 for the record kernel's running maximum
    if (cudaMemcpyAsync(dgrids, G, sizeof G, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dlayer, &L, sizeof L, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(dstatus, 0, sizeof(DevStatus), st) != cudaSuccess ||
        cudaMemsetAsync(counts, 0, csize * (size_t)NA * (size_t)NB, st) != cudaSuccess ||
        cudaMemcpyAsync(dg64, gA, sizeof(double) * NA * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dg64 + NA * d, gB, sizeof(double) * NB * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return QT_ECUDA;
    const long long recs = NApad + NBpad;
    prep_records_kernel<<<(unsigned)((recs + 255) / 256), 256, 0, st>>>(dg64, dgrids, 2, d, rec_floats, 2, recs,
                                                                        drec, nullptr);
    if (cudaGetLastError() != cudaSuccess) return QT_ECUDA;

    ForwardParams fp;
    memset(&fp, 0, sizeof fp);
    fp.d = d;
    fp.n = 1;
    fp.form = kF32Recheck;
    fp.source = kArrays;
    fp.prec = 0;
    fp.counts_u32 = counts_type == QT_COUNTS_U32;
    fp.M = (unsigned long long)M;
    fp.total_items = L.items;
    fp.tile = tile;
    fp.rec_floats = rec_floats;
    fp.rec64_doubles = 2;
    fp.smem_grid_bytes = (int)grid_bytes;
    fp.smem_hist_entries = 0;
    fp.spin_budget = 10000000ll;   // microseconds
    fp.layers = dlayer;
    fp.grids = dgrids;
    fp.g64 = dg64;
    fp.rec32 = drec;
    fp.srcX = X;
    fp.srcY = Y;
    fp.counts = counts;
    fp.cellsA = ii;
    fp.cellsB = jj;
    fp.status = dstatus;
    int bps = 0;
    if (forward_launch(kF32Recheck, dm, S, false, fp, block, (int)grid_bytes, ds.num_sms, &bps, st) !=
        cudaSuccess)
        return QT_ECUDA;

    // report the kernels' status (a copy into a host stack variable, no allocation)
    DevStatus hs;
    if (cudaMemcpyAsync(&hs, dstatus, sizeof hs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QT_ECUDA;
    if (hs.code == QT_ETIMEOUT) return QT_ETIMEOUT;
    if (hs.code != 0) return QT_EDEVICE;
    return QT_OK;
}
