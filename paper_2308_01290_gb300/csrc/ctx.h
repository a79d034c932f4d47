// Host-side solve handle shared by the C ABI and the solver orchestration.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "model_tables.h"
#include "recon.h"

namespace recon {

constexpr int kNumFields = RECON_F_COUNT;
constexpr int kNumSpectra = 3;

struct DevItemList {
    std::vector<Item> h_items;
    std::vector<int> h_lo, h_cnt;
    Item* items = nullptr;
    int* lo = nullptr;
    int* cnt = nullptr;
    double* partials = nullptr;
    unsigned int* counters = nullptr;
    int n = 0;
    int cap = 0;                 // items the device arrays hold
    ItemList view() const { return ItemList{items, n, lo, cnt, partials, counters}; }
};

struct Ctx {
    int n = 0;             // slices
    int precision = 1;     // 1: float maps, 0: double maps
    size_t elem = 4;       // bytes per real element
    cudaStream_t stream = nullptr;
    std::vector<recon_geometry> geo;
    std::vector<recon_params> prm;
    std::vector<Tables> tab;
    std::vector<SliceGeom> sg;
    long long pool_elems = 0;    // real elements per field pool
    long long spec_elems = 0;    // complex elements per spectrum pool
    long long ext_elems = 0;     // unpadded image elements over all slices
    int max_nx = 0, max_ny = 0;
    bool sino_input = false;
    long long sino_elems = 0;
    std::vector<long long> sino_off;

    // device memory
    SliceGeom* d_geom = nullptr;
    SliceConst* d_const = nullptr;
    SliceState* d_state = nullptr;
    void* field[kNumFields] = {};
    void* spec[kNumSpectra] = {};
    float* d_stage[2] = {};      // unpadded float staging (inputs / outputs)
    float* d_sino[2] = {};       // sinogram staging when inputs are sinograms
    float* d_filt = nullptr;     // filtered sinogram scratch (one slice)
    void* d_tw = nullptr;        // FFT twiddle tables (map precision)
    void* d_sym = nullptr;       // |F dx|^2 symbol tables 4 sin^2(pi t/N) (map precision)
    int* d_cg_pending = nullptr; // [0] slices whose Z^m PCG runs, [1] most steps a finished slice took
    int* h_cg_pending = nullptr; // pinned
    int cg_pred = 0;             // steps of the last Z^m solve: when the host first checks the next one

    // accounting: algorithmic bytes per kernel family (device counters) and
    // optional CUDA-event timing of the families in prof_mask
    unsigned long long* d_acct = nullptr;
    unsigned prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    long long fam_launches[KF_COUNT] = {};
    unsigned long long host_acct[KF_COUNT] = {};   // algorithmic bytes of launches accounted on the host

    DevItemList tiles, rows, cols;
    DevItemList tmp_tiles;       // per-slot operations of the serving engine
    // multigrid preconditioner of the Z^m PCG (slices with mg_lb > 0)
    std::vector<int> mg_lb;                   // per slice: tile levels below its own grid (0: FFT preconditioner)
    int mg_max_lb = 0;
    std::vector<std::vector<SliceGeom>> mg_sg;   // [l][s], l >= 1: grid of level l (nx = 0 where absent)
    std::vector<SliceGeom*> d_mg_geom;        // [l]: device copies ([0] = d_geom)
    SliceGeom* d_mg_block = nullptr;          // per slice: its block level (nx = 0: none)
    std::vector<DevItemList> mg_tiles;        // [l], l < mg_max_lb: tiles of level l of the slices with mg_lb > l
    void* mg_pool[3] = {};                    // residual f, a^2 and correction e of the levels >= 1
    int mg_block_smem = 0, mg_inv_smem = 0;
    void* mg_qinv = nullptr;                  // per slice: inverse of its coarsest operator (kMgCoarsePx^2)
    DevItemList pcg_rows, pcg_cols;           // row and column items of the slices on the FFT preconditioner
    DevItemList cg_tiles;                     // k_cg_init tiles: slices without a band fine level
    DevItemList thr_band, thr_tiles;          // threshold pass: band items (FP32, width % 4 == 0, <= 512), tiles of the rest
    std::vector<DevItemList> mg_strips;       // [l]: band items of level l (k_mgb_*; FP32, width % 8 == 0, <= 512)
    std::vector<DevItemList> mg_wide;         // [l]: strip items of the wider such levels (k_mgs_*)
    std::vector<DevItemList> mg_tiles_rest;   // [l]: tile items of level l of the other slices (k_mg_down, k_mg_up)
    int mg_rb = 32;                           // rows a warp walks per strip item on the fine level
    std::vector<int> mg_level_rb;             // per coarse level l >= 1: rows a warp walks per item (0: default)
    int band_res = 0;                         // resident blocks of the coarse band kernels on the device
    std::vector<SliceConst> hconst;
    // serving mode: every slot laid out at capacity; lists hold the active slots
    bool server_mode = false;
    // sinogram-domain data terms (domain 1)
    int domain = 0;
    double gamma = 0.0;             // ||A 1||^2 / (nx ny)
    float* d_sino_tmp = nullptr;    // one sinogram per slice (A p)
    // domain 2 (polyenergetic Gauss-Newton): per ray and slice l1 = A f1, l2 = A f2,
    // W11, W22, v1 / gamma, v2 / gamma (kGnArrays sinograms of n slices each), and
    // the detected spectra of both arms (bins x (w, mu_hat_1, mu_hat_2), float)
    float* d_gn = nullptr;
    float* d_spec = nullptr;
    int spec_nb[2] = {0, 0};
    int cap_nx = 0, cap_ny = 0;
    std::vector<std::pair<int, std::pair<long long, long long>>> tw_index;   // N -> (twiddle, symbol) offsets
    bool has_data = false;
    int cg_parity = 0;
    // side stream of the rho_e FFT solve, which runs beside the Z^m PCG
    // (ordered with `stream` by the two events)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    // host sinograms come in on this stream, one FBP group at a time, while
    // `stream` filters and backprojects the groups before (recon_set_data)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[2] = {nullptr, nullptr};
    // recon_get_async: maps extracted into d_out on `stream`, copied to the host on d2h_stream while the
    // handle goes on with the next inputs (created on the first call)
    cudaStream_t d2h_stream = nullptr;
    cudaEvent_t d2h_ev[2] = {nullptr, nullptr};
    float* d_out[2] = {};
    // one iteration captured as a CUDA graph (recon_set_graph): the Z^m PCG
    // runs as a conditional WHILE node of two PCG steps per body
    bool graph_on = false;
    cudaStream_t graph_stream = nullptr;    // capture and launch stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaEvent_t graph_ev[2] = {nullptr, nullptr};
    int* d_graph_body = nullptr;            // bodies run by the current loop
    unsigned long long* d_graph_launches = nullptr;   // kernels run inside the loops
    long long graph_static_launches = 0;
    // launch shape and row-item size (autotuned on request, recon_set_autotune)
    int grid_mult = 32;          // grid = grid_mult x SMs (grid-stride over items)
    int row_budget = 0;          // complex slots of a row item; 0: the FFT budget
    int autotune = 0;            // 0 off, 1 grid, 2 grid and row-item size
    bool tuned = false;
    long long launches = 0;
    int sm_count = 152;
    std::vector<void*> allocations;
};

// Solver entry points (solver.cu); all queue work on ctx.stream.
int solver_setup(Ctx& c);                      // item lists, constants, scratch
int solver_load_images(Ctx& c, const float* low, const float* high, int on_device);
int solver_init_maps(Ctx& c);
int solver_setup_sino(Ctx& c);                 // domain 1: gamma and the sinogram scratch
int solver_set_graph(Ctx& c, bool on);         // capture each iteration as one CUDA graph
int solver_autotune(Ctx& c);                   // pick grid_mult (and row_budget) by timing
void solver_free_graph(Ctx& c);
long long solver_graph_loop_launches(Ctx& c);  // kernels run inside captured loops so far
int solver_modeb_data(Ctx& c);                 // domain 1: data images t_k from the sinograms
int solver_iterate(Ctx& c, bool stats);        // one iteration of Algorithm 1
int solver_op(Ctx& c, int op);
int solver_extract(Ctx& c, float* Z, float* rhoe, float* f1, float* f2, int on_device);
// the maps of slices s0 .. s1-1 only (outputs indexed as for the whole handle)
int solver_extract_range(Ctx& c, int s0, int s1, float* Z, float* rhoe, float* f1, float* f2);
// two-step comparator maps (device, unpadded) from the loaded pair, or from
// the unpadded images lo, hi (1/mm) when set
int solver_direct(Ctx& c, const float* lo, const float* hi, float* Z, float* rhoe);
int solver_mono(Ctx& c, int n_e, const double* kev, float* out); // monoenergetic images (device, unpadded)
int solver_read_state(Ctx& c, std::vector<SliceState>& out);
int solver_profile_read(Ctx& c, double* ms, long long* launches, unsigned long long* bytes);
// serving engine (slots of a capacity-sized handle)
int solver_configure_slot(Ctx& c, int s, const recon_geometry& g, const recon_params& p);
int solver_rebuild_lists(Ctx& c, const std::vector<int>& active);
int solver_init_slots(Ctx& c, const std::vector<int>& slots, const float* lo, const float* hi);
int solver_extract_slots(Ctx& c, const std::vector<int>& slots, float* Z, float* rhoe);

// Input stage (ct.cu), float device buffers.
int ct_project(const recon_geometry& g, int n, const float* img, float* sino, cudaStream_t st, long long* launches);
// Variants on padded layouts: slice s at img + s * stride, rows pitch apart;
// ct_backproject_add adds A^T sino into img (the caller clears it).
int ct_project_pitched(const recon_geometry& g, int n, const float* img, long long pitch, long long stride,
                       float* sino, cudaStream_t st, long long* launches);
int ct_backproject_add(const recon_geometry& g, int n, const float* sino, float* img, long long pitch,
                       long long stride, cudaStream_t st, long long* launches, const float* wt = nullptr);
int ct_backproject(const recon_geometry& g, int n, const float* sino, float* img, cudaStream_t st,
                   long long* launches);
int ct_fbp(const recon_geometry& g, int n, const float* sino, float* img, float* scratch, cudaStream_t st,
           long long* launches);
// The checks ct_fbp makes before any launch (geometry, shared-memory tables of
// the filter and the backprojection, slice count): RECON_OK or RECON_EINVAL.
int ct_fbp_check(const recon_geometry& g, int n);

// Records CUDA events around the launches of one kernel family when that
// family is selected in Ctx::prof_mask.
struct FamTimer {
    Ctx& c;
    int fam;
    cudaEvent_t b = nullptr, e = nullptr;
    FamTimer(Ctx& ctx, int f);
    ~FamTimer();
};

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define RECON_CUDA(call)                                  \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

}  // namespace recon
