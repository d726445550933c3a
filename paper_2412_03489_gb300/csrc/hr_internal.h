// Host-side internal declarations of libhr (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hr {

// One sample group: P antithetic pairs drawn for one component choice
// (element-wise) or from the mixture (aggregate), stored at perturbations
// [m0, m0 + 2P).  Weight rows of width E start at row m0.
struct SampleGroup {
    int32_t m0;
    int32_t P;
    int32_t lobe;        // 0 gradient lobes, 1 Hessian lobes
    int32_t comp_i;      // -1: aggregate
    int32_t comp_j;
    int32_t quantity;    // 0 grad, 1 hessian, 2 hvp with v, 3 hvp deferred (store n^2/S only),
                         // 4 element-wise hvp of row comp_i (comp_j = -2: row-mixture component)
    uint32_t sub;        // Philox counter word 2 low 24 bits
    uint32_t request;    // Philox counter word 3
    int32_t theta_row;   // which parameter row the group perturbs (multi-instance)
    int32_t pad;
};

struct SampleArgs {
    const SampleGroup* groups;
    int32_t n;
    int32_t E;            // weight row width (0 if no weights written)
    double sigma;
    double Zg, Zd, Zo;
    uint64_t seed;
    const double* v;      // [n] for quantity 2
    float* tau;           // [M][n]
    float* w;             // [M][E] or null
    float* invS;          // [M] n^2 / S (Hessian mixture) or null
    uint2* meta;          // [M] (sub, pair k) or null
    const int32_t* step;  // optional device step index s: every group's sub += 64 s
    const double* sigma_row;  // optional [rows]: group sigma = sigma_row[theta_row] (Z's derived in-kernel)
    int32_t threads;          // threads per block: 16, 32 (0 = 32), 64 or 128; no effect on the results
    // up to kInlineGroups groups passed by value (n_inline > 0: groups[] is not read)
    int32_t n_inline;
    SampleGroup inline_groups[4];
    // optional: the first block also writes theta in FP32 (RN) to theta_out[theta_n],
    // from theta_in (device, FP64) or, when theta_in is null, from theta_vals
    const double* theta_in;
    float* theta_out;
    int32_t theta_n;
    float theta_vals[64];
};
constexpr int kInlineGroups = 4;

void launch_sample(const SampleArgs& a, int n_groups, int max_P, cudaStream_t s);

// g[b][e] = 1/Mg sum of w[m][e] loss[m] over rows [b per_inst, b per_inst + Mg)
// (Kahan FP32 chunks, FP64 tree); grid (n, B)
void launch_grad_reduce(const float* w, const float* loss, int n, int per_inst, int Mg, int B, double* g,
                        cudaStream_t s);

struct FinalizeArgs {
    const float* w;       // [M][E]
    const float* loss;    // [M]
    int32_t E;
    int32_t n;
    int32_t pairs2;       // 2P perturbations per element range
    int32_t elementwise;  // element e sums rows [e*2P, (e+1)*2P), else [0, 2P)
    int32_t hessian;      // also write the symmetric n x n matrix
    double inv2P;
    double* out_flat;     // [E]
    double* out_scale;    // [E] or null
    double* out_full;     // [n][n] or null
};
void launch_finalize(const FinalizeArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// render batches: perturbation m renders at RN32(theta32[row(m)] + tau[m])
// ---------------------------------------------------------------------------
// One request's slice of a batched launch (continuous batching): items
// [start, start + count) of the launch render perturbations
// [m_begin, m_begin + count) of that request.
struct BatchRow {
    const float* theta32;   // [n]
    const float* tau;       // [M][n]
    const uint2* meta;      // [M]
    float* loss;            // [M]
    uint64_t seed;
    uint32_t request;
    int32_t m_begin;
    int32_t start;
    int32_t pad;
};
constexpr int kMaxBatchRows = 48;

struct RenderBatch {
    const float* theta32;   // [rows][n]
    const float* tau;       // [M][n]
    const uint2* meta;      // [M] (sub, k): path random numbers (path tracer)
    float* loss;            // [M]
    int32_t M;              // items in this launch
    int32_t n;
    int32_t per_row;        // perturbations per theta row
    uint32_t request0;      // request id of row 0 (row r: request0 + r)
    uint64_t seed;
    int32_t table_rows;     // > 0: items map through `rows` instead
    int32_t pad;
    BatchRow rows[kMaxBatchRows];
};

// the perturbation behind item i of a launch
struct Pert {
    const float* theta;
    const float* tau;
    const uint2* meta;
    float* loss;
    uint64_t seed;
    uint32_t request;
};

#ifdef __CUDACC__
__device__ __forceinline__ Pert resolve(const RenderBatch& b, int i) {
    Pert p;
    if (b.table_rows > 0) {
        int r = 0;
        while (r + 1 < b.table_rows && b.rows[r + 1].start <= i) ++r;
        const int m = b.rows[r].m_begin + (i - b.rows[r].start);
        p.theta = b.rows[r].theta32;
        p.tau = b.rows[r].tau + (size_t)m * b.n;
        p.meta = b.rows[r].meta + m;
        p.loss = b.rows[r].loss + m;
        p.seed = b.rows[r].seed;
        p.request = b.rows[r].request;
    } else {
        const int row = i / b.per_row;
        p.theta = b.theta32 + (size_t)row * b.n;
        p.tau = b.tau + (size_t)i * b.n;
        p.meta = b.meta ? b.meta + i : nullptr;
        p.loss = b.loss + i;
        p.seed = b.seed;
        p.request = b.request0 + (uint32_t)row;
    }
    return p;
}
#endif

struct DevScene;
void launch_render_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s);
// one image at params (FP32 [n]) -> img [H][W][C]
void launch_render_image(const DevScene& sc, const float* d_params, uint64_t seed, uint32_t request,
                         uint32_t sub, uint32_t k, uint32_t tag, int spp, float* d_img, cudaStream_t s);

struct DevScene {
    int kind = 0, W = 0, H = 0, C = 0, n = 0;
    float* target = nullptr;      // [H][W][C]
    // disc
    float radius = 0.f;
    uint32_t* tbits = nullptr;    // [H][(W + 31) / 32] bit-packed target (bit set: pixel is 1)
    int* trowpop = nullptr;       // [H + 1] prefix sums of the packed rows' popcounts
    int tbinary = 0;              // 1: every target pixel is 0 or 1 (the loss is a mismatch count)
    // revolve
    float* verts = nullptr;       // [nv][3]
    int32_t* tris = nullptr;      // [nt][3]
    float* tnrm = nullptr;        // [nt][3] unit model-space normals (FP32)
    float* tile_t2 = nullptr;     // [tiles] sum of target^2 per 8x8 tile
    int nv = 0, nt = 0;
    float albedo[3] = {0, 0, 0}, light[3] = {0, 0, 0};
    float eye_dist = 0.f, scale = 0.f;
    size_t rv_smem = 0;           // dynamic shared memory of one render
    int rv_cap = 0, rv_vreg = 0;  // bin entry capacity, vertex-region floats
    int rv_th = 8;                // raster tile height (8 x rv_th pixel tiles)
    size_t rv_csmem = 0;          // compact layout (two renders per SM): shared memory, 0 = none
    int rv_ccap = 0, rv_cslots = 0;   // its bin entry capacity and survivor slots
    unsigned long long* rv_stats = nullptr;   // [1] renders that took the bin-overflow path
    // tris2d
    float* raw = nullptr;         // [n_tris][9]
    int32_t* pidx = nullptr;      // [n]
    int n_tris = 0;
    // ptbox
    int32_t qaxis[13] = {};
    float qgeom[13][5] = {};
    float qalb[13][3] = {};
    float sc_[3][3] = {}, sr[3] = {}, salb[3][3] = {};
    float light_half = 0.f, cam_z = 0.f, tan_half = 0.f, pix_scale = 0.f;
    float emission[3] = {0, 0, 0};
    int spp = 0, target_spp = 0, depth = 0;
    uint64_t scene_seed = 0;
    unsigned long long* pt_stats = nullptr;   // [4] work counters of the counting launches
    int count_work = 0;                       // 1: path-tracer launches count their rays
    // analytic test functions
    double* qA = nullptr;         // [n][n] FP64 (QUADRATIC)
    double* qb = nullptr;         // [n] FP64
    double gauss_sigma = 0.0;     // NEGGAUSS
    // launch shapes picked by the autotuner; none of them changes a result
    int render_variant = 0;       // index into render_variant_count(kind)
    int sample_threads = 32;
};

// launch-shape variants of a scene kind's render+loss kernel (1 = none)
int render_variant_count(int kind);

// shared-memory layout and tile height of one mesh render on a device with
// max_smem bytes of opt-in shared memory per block (sets rv_smem, rv_cap,
// rv_vreg, rv_th) and, where it fits, of the compact layout that puts two
// renders on an SM (rv_csmem, rv_ccap, rv_cslots); false if the mesh does
// not fit
bool revolve_layout(DevScene& sc, int max_smem, int smem_per_sm);
int revolve_tiles(const DevScene& sc);
void revolve_prepare(DevScene& sc, cudaStream_t s);   // normals, kernel attributes
void revolve_tile_t2(DevScene& sc, cudaStream_t s);   // after the target exists
// disc and squares scenes, after the target exists: sc.tbits, sc.trowpop and sc.tbinary
cudaError_t disc_prepare_target(DevScene& sc, cudaStream_t s);

int num_sms();

}  // namespace hr
