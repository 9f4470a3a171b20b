// qt_internal.h -- structures shared by the host side of libqt and its kernels.
#pragma once
#include <cstdint>

namespace qt {

constexpr int kDMax = 16;          // largest state dimension
constexpr int kChunk = 16;         // candidates per min-tracking chunk of the FP32 screen
constexpr int kSlots = 2;          // ring slots of the streamed-grid mode

enum Form : int32_t { kPlainF64 = 1, kF32Recheck = 2, kTcRecheck = 3, kRouterCert = 4, kPathwise = 5 };
enum Source : int32_t { kSampler = 0, kArrays = 1 };

// Per-layer sampler parameters packed by the host: m[d], b[d], L[d*d], A[d*d],
// T[d*d] (read by every form) and alpha[d], beta[d] (the Euler-scheme chain of
// the path-wise form), padded to a multiple of 4 entries.
__host__ __device__ constexpr int param_stride(int d) { return (4 * d + 3 * d * d + 3) / 4 * 4; }

// Device status block, zeroed before every forward call.
struct DevStatus {
    int32_t code;                  // qt_status of the first error seen, 0 = none
    int32_t where;                 // small tag of the failing site (diagnostics)
    unsigned long long queue;      // persistent work-queue counter
    unsigned long long rechecks;   // FP64 re-evaluations
    unsigned long long candidates; // candidate distances (router form)
    unsigned long long done_items; // work items finished
    unsigned long long spare[4];   // [0]: router grid checksum; [1..3]: diagnostics
};

// One layer pair (k, k+1) of the forward step.
struct LayerDesc {
    int32_t NA, NB;                // grid sizes N_k, N_{k+1}
    int32_t NApad, NBpad;          // sizes padded to a whole number of chunks
    int32_t gridA, gridB;          // grid indices (k, k+1): index into the per-grid tables
    int32_t segA, segB;            // streamed mode: segments per grid (0 = resident)
    long long goffA, goffB;        // point offsets into the FP64 grids
    long long roffA, roffB;        // record offsets (in records) into the prepared grids
    long long coff;                // entry offset of the count block
    long long item_begin;          // first work item of this layer
    int32_t items;                 // work items (sample tiles) of this layer
    int32_t hist_smem;             // 1 = shared-memory privatised histogram for this layer
};

// Per-grid tables written by the preparation kernel.
struct GridInfo {
    float mu[kDMax];               // centre (FP32) subtracted before the screen
    float R;                       // max norm of the centred FP32 records (rounded up)
    int32_t N, Npad;
    long long goff, roff;
    int32_t tc_exp;                // tensor-core form: operands scaled by 2^tc_exp
    int32_t tc_tiles;              // tensor-core form: 256-point operand tiles of this grid
    long long tc_toff;             // tensor-core form: first tile of this grid
};

constexpr int kTcTileN = 256;      // grid points per tensor-core operand tile (MMA N)
constexpr int kTcTileM = 128;      // samples per tensor-core work item (MMA M)
constexpr int kTcThreads = 512;    // tensor-core form: 16 warps (8 epilogue, 2 MMA, tile loader, draw, 4 certifier)
constexpr int kTcMaxSlots = 16;    // tensor-core form: most operand tiles held in shared memory

// Bytes of one work item's drawn samples in the tensor-core form, as the
// certifier warps draw them into an item slot in shared memory, or the draw
// pass writes them to device memory: the FP16 operand rows of both grids
// (128 x K each, core-matrix layout), then the centred FP32 coordinates and
// norms ([grid][dm + 1][128]).
__host__ __device__ constexpr long long tc_item_op_bytes(int K) { return 2ll * kTcTileM * K * 2; }
__host__ __device__ constexpr long long tc_item_cert_bytes(int dm) { return 2ll * (dm + 1) * kTcTileM * 4; }

// Dynamic shared memory of the tensor-core form besides its ring of operand
// tiles (dimension class dm, K columns per operand row).
__host__ __device__ constexpr long long tc_fixed_smem(int dm, int K)
{
    return 2 * tc_item_op_bytes(K)                           // sample operands: 2 items
           + 2ll * 2 * 2 * 5 * kTcTileM * 4                  // chunk states: 2 items x 2 grids x 2 warpgroups x 5
           + 2 * tc_item_cert_bytes(dm);                     // centred samples: 2 items
}

struct ForwardParams {
    // problem
    int32_t d, n;
    int32_t form;                  // Form
    int32_t source;                // Source
    int32_t prec;                  // 0 = FP64 samples, 1 = FP32 samples
    int32_t counts_u32;            // 1 = uint32 counts, 0 = int64
    unsigned long long M;          // samples per layer
    unsigned long long seed;
    long long total_items;
    int32_t tile;                  // samples per work item
    int32_t rec_floats;            // floats per FP32 record (d+1 rounded up to 4)
    int32_t rec64_doubles;         // doubles per FP64 record (d rounded up to 2)
    int32_t smem_grid_bytes;       // bytes of dynamic smem reserved for grids
    int32_t smem_hist_entries;     // u32 entries reserved for the private histogram
    int32_t seg_records;           // streamed mode: records per ring slot (multiple of kChunk)
    long long spin_budget;         // bound of every device wait in microseconds; < 0: give up at once
    int32_t pathwise_euler;        // Algorithm II: 1 = Euler-scheme chain (innovation rows scaled)
    // tables
    const LayerDesc* layers;
    const GridInfo* grids;
    const float* params_f;         // [n][param_count(d)]
    const double* params_d;        // [n][param_count(d)]
    int32_t params_stride;
    // data
    const double* g64;             // FP64 grids [sum N][d] (the exact distances)
    const float* rec32;            // FP32 records [sum Npad][rec_floats]
    const double* rec64;           // FP64 records [sum Npad][rec64_doubles]
    const double* srcX;            // Source::kArrays: samples [M][d]
    const double* srcY;
    void* counts;
    int32_t* cellsA;               // Source::kArrays: optional per-sample cells
    int32_t* cellsB;
    // dump
    long long dump_count, dump_stride;
    double* dumpX;
    double* dumpY;
    int32_t* dumpI;
    int32_t* dumpJ;
    DevStatus* status;
    // tensor-core form
    const void* tc_tiles;          // FP16 operand tiles [tiles][256][K] in the canonical K-major layout
    int32_t tc_k;                  // 16 or 32
    int32_t tc_slots;              // ring slots of operand tiles in shared memory
    int32_t tc_resident;           // 1: both grids' tiles stay in shared memory for the layer
    long long item_lo, item_hi;    // tensor-core form: work items [item_lo, item_hi) of this launch
    int32_t tc_draw_in;            // tensor-core form: 1 = the screen kernel draws its samples
    unsigned char* tc_items;       // tensor-core form, draw pass: samples of the launch's items
    // learned router + Elkan certificate
    const float* rt_params;        // MLP parameters, packed W1, b1, W2, b2, W3, b3
    const float* rt_linv;          // [n+1][d][d] FP32 inverse Cholesky factors (whitening)
    const int32_t* rt_bstart;      // [65] bucket starts into rt_members
    const int32_t* rt_members;     // [N] grid indices sorted by bucket
    const int32_t* rt_nb_idx;      // [n+1][N][C] neighbours of each grid point, nearest first
    const float* rt_nb_dist;       // [n+1][N][C] their distances, rounded down
    int32_t rt_C;                  // neighbours per point
    int32_t rt_N;                  // common grid size of layers >= 1
    unsigned long long rt_checksum;// checksum of the grids the router was built for
};

constexpr int kSwingQ = 8;         // swing option: consumption states per warp

constexpr int kRtHidden = 64;      // router MLP width
constexpr int kRtBuckets = 64;     // router classes (buckets of grid points)
__host__ __device__ constexpr int rt_param_count(int d) { return kRtHidden * d + kRtHidden + 2 * (kRtHidden * kRtHidden + kRtHidden); }

}  // namespace qt
