// Internal declarations of the gbfwi library (sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "gbfwi.h"
#include "ptrclass.h"

#define GB_NG 5

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------

#define GB_CUDA(call)                                                    \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) {                                         \
            gb_set_last_cuda_error(_e, #call, __FILE__, __LINE__);       \
            return GBFWI_ECUDA;                                          \
        }                                                                \
    } while (0)

#define GB_TRY(expr)                    \
    do {                                \
        int _rc = (expr);               \
        if (_rc != GBFWI_OK) return _rc; \
    } while (0)

void gb_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);
// records what was non-finite (named by gbfwi_strerror) and returns GBFWI_ENONFINITE
int gb_nonfinite(const char *what);
void gb_note_launch();
void gb_note_launches(long long n);        // kernels launched by a graph replay
long long gb_launches_so_far();

// after every kernel launch: count it and surface launch errors
#define GB_LAUNCHED()                 \
    do {                              \
        gb_note_launch();             \
        GB_CUDA(cudaGetLastError());  \
    } while (0)

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t nbytes);          // grow-only cudaMalloc
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

// GB_PTR_HOST, GB_PTR_LOCAL or GB_PTR_FOREIGN for a caller's array (NULL is host)
int gb_ptr_class(const void *ptr);
// true when ptr is memory of the current device (or managed memory)
bool gb_is_device_ptr(const void *ptr);

// GBFWI_OK when every given array is host memory or memory of the current
// device; GBFWI_EINVAL when one lives on another device (the kernels would
// fault on it instead of returning an error)
inline int gb_check_local() { return GBFWI_OK; }
template <class P, class... Rest>
int gb_check_local(P p, Rest... rest)
{
    if (gb_ptr_class(static_cast<const void *>(p)) == GB_PTR_FOREIGN) return GBFWI_EINVAL;
    return gb_check_local(rest...);
}

// ---------------------------------------------------------------------------
// element tiles
// ---------------------------------------------------------------------------

struct TileShape { int tx, tz; };
static constexpr int kNumTiles = 5;
extern const TileShape kTiles[kNumTiles];

// injection entry: F_x += wx * sig[cx], F_z += wz * sig[cz]
struct InjEntry { int cx, cz; float wx, wz; };
// entries [begin, end) all act on owned node (ox, oz) of the tile, packed
// as node = oz * (4 TX + 1) + ox
struct InjGroup { int node, begin, end, pad; };

struct TileLists {
    bool built = false;
    int ntx = 0, ntz = 0;
    DevBuf src_gptr;     // int [nsrc][ntiles + 1]
    DevBuf src_groups;   // InjGroup
    DevBuf src_entries;  // InjEntry
    DevBuf rec_gptr;     // int [ntiles + 1]   (adjoint sources at the receivers)
    DevBuf rec_groups;
    DevBuf rec_entries;
    DevBuf rec_tptr;     // int [ntiles + 1]   receivers recorded by each tile
    DevBuf rec_list;     // int receiver ids, grouped by tile
};

// ---------------------------------------------------------------------------
// mesh handle
// ---------------------------------------------------------------------------

struct gbfwi_mesh {
    gbfwi_mesh_desc d{};
    int nx = 0, nz = 0, pitch = 0;      // node grid; pitch = row length in nodes (multiple of 4)
    double xi[GB_NG], w[GB_NG], D[GB_NG][GB_NG];
    std::vector<gbfwi_source> src;
    std::vector<double> rec_xz;
    int nrec = 0;
    // receivers: element and 25 interpolation weights
    std::vector<int> rec_ex, rec_ez;
    std::vector<float> rec_w;            // [nrec][25], index j*5+i
    // sources: nodal weights
    struct SrcNode { int ix, iz; float wx, wz; };
    std::vector<std::vector<SrcNode>> src_nodes;
    // assembled 1-D quadrature weights (metres): W_g = wx[ix] * wz[iz]
    std::vector<double> wx1, wz1;
    gbfwi_schedule sch{1, 0, 0, 0, 1};
    bool have_model = false;
    double dx_min = 0;                   // smallest GLL node spacing

    // device tables
    DevBuf d_lm;        // float2 [nz][pitch]  (lambda, mu)
    DevBuf d_minv;      // float  [nz][pitch]  1 / M
    DevBuf d_bnd;       // float4 [nz][pitch]  (Cx, Cz, 1/(M + dt/2 Cx), 1/(M + dt/2 Cz)); edges only
    DevBuf d_bw;        // float4 [nz][pitch]  (Wn_x, Wn_z, Wt_x, Wt_z) Stacey edge weights
    DevBuf d_model;     // float  [3][nz][pitch] rho, vp, vs
    DevBuf d_wx, d_wz;  // float  [nx], [nz]
    DevBuf d_recw;      // float  [nrec][25]
    DevBuf d_rec_e;     // int2   [nrec] element (ex, ez)
    DevBuf d_stf;       // float  [nsrc][nt + 1]
    TileLists lists[kNumTiles];

    // work buffers (grown on demand)
    DevBuf w_hist, w_vh, w_adj, w_wh, w_acc, w_snap, w_seis, w_sig, w_obs, w_grad,
        w_red, w_flag, w_shots, w_tmp, w_stage;
    DevBuf w_pc;        // preconditioner accumulators
    DevBuf w_status;    // int: nonzero after a step kernel's bounded wait gave up

    DevBuf w_batch;     // shot ids of the batch being replayed (fixed address for graphs)
    DevBuf w_lacc;      // gradient accumulators of the batch in flight (fixed address for graphs)
    // extra concurrent lanes of adjoint_gradient (lane 0 uses the buffers above)
    struct Lane {
        DevBuf hist, snap, vh, adj, wh, seis, batch, acc;
        cudaStream_t st = nullptr;
        ~Lane() { if (st) cudaStreamDestroy(st); }
    };
    std::vector<Lane *> lanes;
    // CUDA graphs of whole forward / adjoint passes, keyed by schedule,
    // batch size and work-buffer addresses
    struct CachedGraph {
        std::string key;
        cudaGraphExec_t exec;
        long long kernels;   // kernel launches recorded while capturing
    };
    std::vector<CachedGraph> graphs;
    cudaStream_t cap_stream = nullptr;

    // optional per-phase timing of adjoint_gradient
    bool timing = false;
    std::vector<cudaEvent_t> ev;        // 4 per shot batch
    int ev_used = 0;
    long long fwd_launches = 0, adj_launches = 0;
    bool timed_valid = false;
    double fwd_ms = 0, adj_ms = 0;
    ~gbfwi_mesh();
};

int gb_build_tile_lists(gbfwi_mesh *m, int tile);
// after the work on the mesh has completed: GBFWI_ETIMEOUT (and the flag
// cleared) when a step kernel's bounded wait gave up since the last check
int gb_take_status(gbfwi_mesh *m);

// ---------------------------------------------------------------------------
// kernel argument block of the time step (one launch = one step of every
// shot of a batch)
// ---------------------------------------------------------------------------

enum StepMode { MODE_FWD = 0, MODE_FWD_PC = 1, MODE_ADJ_G = 2, MODE_ADJ_PC = 3 };

struct StepArgs {
    int nex, nez, nx, nz, pitch;
    float dt;
    long long fstride;            // float2 elements between shots of every field
                                  // (fields are stored [slot][shot][nz][pitch])
    const float2 *ucur;           // u_{n+1} (read, window)
    float2 *unext;                // u_{n+2} (written, owned nodes)
    float2 *vh;                   // half-step velocity, in place (owned nodes)
    const float2 *uold;           // level n of the same field (P-modes)
    long long hstride;            // float2 elements between shots of the history (= fstride)
    const float2 *h0, *h1, *h2;   // forward history levels (adjoint modes)
    const float2 *lm;
    const float *minv;
    const float4 *bnd;
    const float4 *bw;
    const float *wxs, *wzs;
    // injection
    const int *gptr; const InjGroup *groups; const InjEntry *entries;
    int per_shot_groups;          // 1: groups indexed by source id
    int ntiles;
    const float *sig; long long sig_shot_stride; int sig_chan_stride; int tsig; float sig_scale;
    const int *shot_map;          // batch slot -> source id (or nullptr: identity)
    // recording
    const int *rec_tptr, *rec_list; const float *recw; const int2 *rec_e;
    float *seis; long long seis_shot_stride; int nt; int trec;
    // accumulators
    float *acc; long long acc_shot_stride; long long acc_comp_stride;
    // set to 1 when a bounded device-side wait gave up (the step's results are invalid)
    int *status;
};

int gb_launch_step(int mode, int tile, const StepArgs &a, int nbatch, cudaStream_t s);
int gb_prepare_step(int mode, int tile);   // set kernel attributes outside any stream capture

// small kernels of the SEM driver
int gb_material(gbfwi_mesh *m, cudaStream_t s);

// tensor-core products of the BFGS / randomized-SVD blocks
// (tc_products.cu).  Rows are length-n FP32 vectors with row stride ld (a
// multiple of 64 floats; rows 256-byte aligned, readable up to the pitch);
// an operand of ka rows takes rows a < ka1 from A1 and the rest from A2
// (likewise B).
//   out[a][b] (FP64, row stride ldo) = sum_i A_a[i] B_b[i], through
//   gb_tc_atb_splits(ka, kb, n) * ka * kb doubles of split-K partials
//   (tcgen05; *status set to 1 when a bounded wait gave up);
//   out[c][i] = sum_a coef[c][a] R_a[i] + beta dw[i] Xc[c][i] (ktot <= 128;
//   tcgen05, same status flag).
long long gb_tc_atb_splits(int ka, int kb, long long n);
int gb_tc_atb(const float *A1, const float *A2, int ka1, int ka, const float *B1, const float *B2, int kb1, int kb,
              long long ld, long long n, double *part, size_t part_doubles, double *out, long long ldo,
              int *status, cudaStream_t s);
int gb_tc_combine(const float *R1, const float *R2, int k1, int ktot, long long ldr, const float *coef, int nc,
                  long long n, float *out, long long ldo, const float *dw, const float *Xc, long long ldx,
                  float beta, int *status, cudaStream_t s);
