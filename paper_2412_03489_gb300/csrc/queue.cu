// K10: persistent serving queue (hr_queue_*): many small estimate requests on
// a disc or squares scene served by one long-running launch.
//
// Submission costs no driver call.  The host writes a request's descriptor
// into a ring in host-mapped memory and then release-stores the count of
// submitted requests.  Inside the kernel:
//   - one dispatcher warp polls that count, copies new descriptors into a
//     device ring, writes each new work unit's (request, unit) pair into a
//     device unit ring and publishes the count of units;
//   - every other warp takes a ticket, one atomicAdd on a claim counter, and
//     runs the unit with that index once it is published.
// A unit is 16 antithetic pairs of one request; the warp that holds it
// (1) samples the 32 perturbations, one pair leg per lane, with the sampler's
// code (Sec. 3.2-3.5), (2) renders each of them with the scene's renderer
// fused with the L2 loss (the plain kernels' code), one warp per render, and
// (3) counts the unit as finished.
// The warp that finishes a request's last unit forms the estimator sums in the
// sum kernel's order: 256 Kahan chunks, then the same FP64 tree.  It writes
// the result and a completion flag to host-mapped memory.  A request's
// result is therefore bit-identical to hr_estimate_* with the same options.
//
// Waits are bounded.  The dispatcher leaves after idle_budget_us of clock64()
// time without a new request and then tells the workers to leave.  A worker
// that sees neither a new unit nor that word for longer than a larger safety
// bound leaves on its own.  The last warp to leave rewinds the claim counter
// to the published count (tickets taken past it were never run) and writes
// the exit code to a status word in host-mapped memory: HR_ERR_TIMEOUT after
// an idle exit, HR_OK after a stop.  The host launches the kernel again when
// work arrives after an exit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "disc_device.cuh"
#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"
#include "sample_device.cuh"

namespace hr {
namespace {

constexpr int kQWarps = 8;           // warps per CTA
constexpr int kQPairs = 16;          // antithetic pairs per work unit
constexpr int kQMaxN = 8;            // parameters of a queued request
constexpr int kQMaxGroups = 4;       // sample groups of a queued request
constexpr int kQMaxResult = kQMaxN * kQMaxN;
constexpr int kQUnitBits = 24;       // unit ring entry = request << 24 | unit
constexpr unsigned long long kQUnitMask = (1ull << kQUnitBits) - 1ull;
constexpr int kQUnitRing = 1 << 20;  // unit ring entries
constexpr int kQReplicas = 8;        // device copies of each descriptor (unit k reads copy k % 8)
constexpr int kQBatch = 4;           // descriptors the dispatcher loads per pass

// The sampler's inputs of a request (the fields sample_leg reads).
struct QSample {
    int32_t n, E;
    uint64_t seed;
    const double* v;                 // set to QReq::vv on the device
    float* tau;                      // [G M][n]
    float* w;                        // [G M][E]
    float* invS;                     // null
    uint2* meta;                     // null
    const int32_t* step;             // null
};

struct __align__(16) QReq {
    QSample sa;
    Lobes lobes;
    SampleGroup groups[kQMaxGroups];
    double vv[kQMaxN];               // HVP direction
    float theta32[kQMaxN];           // theta rounded to FP32
    float* loss;                     // [G M] losses
    double* res;                     // host-mapped result (n or n*n doubles)
    int* flag;                       // host-mapped completion flag
    unsigned* done;                  // units finished (device; reset by the finishing warp)
    int units, G, P, E, n, elementwise, hessian, pad;
    double inv2P;
};

// one 16-byte load per lane copies a descriptor
static_assert(sizeof(QReq) <= 32 * 16, "a queue descriptor is at most 512 bytes");
constexpr int kQInt4 = (int)(sizeof(QReq) / 16);

// Device control block; the claim counter (atomics) and the published counts
// (polled by idle warps) sit on separate 128-byte lines.
struct QCtl {
    alignas(128) unsigned long long claim;   // next ticket
    alignas(128) unsigned long long units;   // units published (dispatcher, release)
    unsigned long long reqs;                 // requests copied into the device ring
    alignas(128) int running;                // warps still in the kernel (set at launch)
    int stop;                                // dispatcher: workers leave once idle (reset at launch)
    int code;                                // first non-zero exit code of this launch (reset at launch)
};

// Host-mapped control block.
struct QHost {
    unsigned long long submitted;    // requests written into the host ring (host, release store)
    int stop;                        // host: leave once the queue is empty
    int status;                      // 1 while a launch runs, then its exit code
};

struct QArgs {
    QCtl* ctl;
    QHost* host;                     // device view of the host-mapped block
    const QReq* h_ring;              // device view of the host ring
    QReq* d_ring;                    // [cap][kQReplicas]
    unsigned long long* unit_ring;   // [kQUnitRing] request << 24 | unit
    int cap;                         // request ring slots
    int W, H;
    float radius;
    const float* target;
    DiscBits tb;                     // bit-packed binary target (bits null: not binary)
    long long budget;                // dispatcher idle budget, clock64 cycles
    long long safety;                // worker wait bound, clock64 cycles
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(int* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Estimator sums of one request by one warp, in the order of the sum kernel:
// element e sums its 2P rows as 256 contiguous chunks, each a Kahan FP32 sum
// of w * loss, then the pairwise FP64 tree (t, t + o) for o = 128, 64, 32 and
// a shuffle tree over the last 32; lane l holds chunks l + 32 j, j = 0..7.
__device__ void queue_finalize(const QReq& R, int lane) {
    const int cnt = 2 * R.P;
    const int chunk = (cnt + 255) / 256;
    for (int e = 0; e < R.E; ++e) {
        const int m0 = R.elementwise ? e * cnt : 0;
        double h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b = m0 + (lane + 32 * j) * chunk;
            const int end = min(m0 + cnt, b + chunk);
            Kahan ks;
            for (int m = b; m < end; ++m)
                ks.add(__fmul_rn(__ldcg(R.sa.w + (size_t)m * R.E + e), __ldcg(R.loss + m)));
            h[j] = (double)ks.s - (double)ks.c;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] += h[j + 4];
        h[0] += h[2];
        h[1] += h[3];
        h[0] += h[1];
        double vs = h[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vs += __shfl_down_sync(0xffffffffu, vs, o);
        if (lane == 0) {
            const double val = vs * R.inv2P;
            if (R.hessian) {
                int r = 0, rem = e;
                while (rem >= R.n - r) { rem -= R.n - r; ++r; }
                const int c = r + rem;
                R.res[r * R.n + c] = val;
                R.res[c * R.n + r] = val;
            } else {
                R.res[e] = val;
            }
        }
    }
}

// The dispatcher: moves descriptors from the host ring to the device ring and
// lists their units in the unit ring.  Returns the exit code.
__device__ int dispatch_loop(const QArgs& A, int lane) {
    unsigned long long seen = ld_acquire_gpu(&A.ctl->reqs);
    unsigned long long U = ld_acquire_gpu(&A.ctl->units);
    long long t0 = clock64();
    unsigned ns = 64;
    for (;;) {
        unsigned long long hs = 0;
        int stop = 0;
        if (lane == 0) {
            hs = ld_acquire_sys(&A.host->submitted);
            stop = ld_volatile(&A.host->stop);
        }
        hs = __shfl_sync(0xffffffffu, hs, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (hs > seen) {
            // kQBatch descriptors per pass: their host-memory loads are in
            // flight together; each is stored as kQReplicas device copies on
            // different lines, so that the warps taking one request's units
            // spread their loads over the L2
            for (unsigned long long r0 = seen; r0 < hs; r0 += kQBatch) {
                const int cnt = (int)min((unsigned long long)kQBatch, hs - r0);
                int4 v[kQBatch];
                int un[kQBatch];
#pragma unroll
                for (int j = 0; j < kQBatch; ++j) {
                    if (j >= cnt) break;
                    const int slot = (int)((r0 + j) % (unsigned long long)A.cap);
                    if (lane < kQInt4) v[j] = __ldcv(reinterpret_cast<const int4*>(A.h_ring + slot) + lane);
                    un[j] = __ldcv(&A.h_ring[slot].units);
                }
#pragma unroll
                for (int j = 0; j < kQBatch; ++j) {
                    if (j >= cnt) break;
                    const unsigned long long r = r0 + j;
                    const int slot = (int)(r % (unsigned long long)A.cap);
                    if (lane < kQInt4)
                        for (int c = 0; c < kQReplicas; ++c)
                            __stcg(reinterpret_cast<int4*>(A.d_ring + (size_t)slot * kQReplicas + c) + lane, v[j]);
                    for (int k = lane; k < un[j]; k += 32)
                        __stcg(A.unit_ring + ((U + (unsigned long long)k) % kQUnitRing), (r << kQUnitBits) | (unsigned)k);
                    U += (unsigned long long)un[j];
                }
                // publish each pass, so that workers start on a long backlog
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    st_release_gpu(&A.ctl->reqs, r0 + (unsigned long long)cnt);
                    st_release_gpu(&A.ctl->units, U);
                }
            }
            seen = hs;
            t0 = clock64();
            ns = 64;
            continue;
        }
        if (stop) return HR_OK;
        if (clock64() - t0 > A.budget) return HR_ERR_TIMEOUT;
        __nanosleep(ns);
        ns = min(2u * ns, 2048u);
    }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Ticket u: 1 when its unit is published (acquired), 0 when it will not be
// (block: the dispatcher stopped with u at or past the final count; !block:
// not yet published), -1 when a blocking wait passed the safety bound without
// any newly published unit.  Every lane returns the same value.
__device__ int ticket_wait(const QArgs& A, int lane, unsigned long long u, bool block) {
    int got = 0;
    if (lane == 0) {
        if (!block) {
            got = u < ld_acquire_gpu(&A.ctl->units) ? 1 : 0;
        } else {
            long long t0 = clock64();
            unsigned long long last = ~0ull;
            unsigned ns = 128;
            for (;;) {
                const unsigned long long pub = ld_acquire_gpu(&A.ctl->units);
                if (u < pub) { got = 1; break; }
                if (pub != last) {
                    last = pub;
                    t0 = clock64();
                }
                if (ld_acquire_gpu(&A.ctl->stop)) {
                    // the count read after stop is final: a ticket below it still runs
                    if (u < ld_acquire_gpu(&A.ctl->units)) got = 1;
                    break;
                }
                if (clock64() - t0 > A.safety) { got = -1; break; }
                __nanosleep(ns);
                ns = min(2u * ns, 4096u);
            }
        }
        if (got > 0) __threadfence();
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, got, 0);
}

// Start copying the descriptor of published ticket u into dst (completed by
// cp_async_wait_all); returns the unit's index within its request.
__device__ __forceinline__ int fetch_desc(const QArgs& A, int lane, unsigned long long u, QReq* dst) {
    const unsigned long long ent = __ldcg(A.unit_ring + (u % kQUnitRing));
    const int slot = (int)((ent >> kQUnitBits) % (unsigned long long)A.cap);
    const int unit = (int)(ent & kQUnitMask);
    const int4* src = reinterpret_cast<const int4*>(A.d_ring + (size_t)slot * kQReplicas + unit % kQReplicas);
    if (lane < kQInt4) cp_async16(reinterpret_cast<int4*>(dst) + lane, src + lane);
    return unit;
}

// kKind: HR_SCENE_DISC2D or HR_SCENE_BOXES2D (the renders of the plain kernels)
template <int kKind>
__global__ void __launch_bounds__(32 * kQWarps, 3) queue_kernel(QArgs A) {
    __shared__ float s_px[HR_MAX_IMAGE_SIDE], s_py[HR_MAX_IMAGE_SIDE];
    __shared__ float s_c[kQWarps][kQMaxN];   // squares: the perturbed centres of the current render
    __shared__ int s_sp[kQWarps][kQMaxN];    // squares: their column intervals
    __shared__ QReq s_req[kQWarps][2];
    centre_tables(s_px, s_py, A.W, A.H);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int code = HR_OK;
    if (blockIdx.x == 0 && warp == 0) {
        code = dispatch_loop(A, lane);
        // no more units get published: the workers leave once they run out
        // (stop is released after the last published count)
        if (lane == 0) st_release_gpu(&A.ctl->stop, 1);
    } else {
        // Two descriptor buffers per warp: while one unit is sampled and
        // rendered, the next ticket's descriptor (when already published)
        // is on its way into the other buffer.
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(&A.ctl->claim, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        int got = ticket_wait(A, lane, u, true);
        int cur = 0;
        int unit = got > 0 ? fetch_desc(A, lane, u, &s_req[warp][0]) : 0;
        while (got > 0) {
            cp_async_wait_all();
            __syncwarp();
            QReq& R = s_req[warp][cur];
            if (lane == 0) R.sa.v = R.vv;
            __syncwarp();
            // the next ticket; its descriptor is fetched now if it is published
            unsigned long long un = 0;
            if (lane == 0) un = atomicAdd(&A.ctl->claim, 1ull);
            un = __shfl_sync(0xffffffffu, un, 0);
            const int ready = ticket_wait(A, lane, un, false);
            int unit_n = ready > 0 ? fetch_desc(A, lane, un, &s_req[warp][1 - cur]) : 0;
            // 1. sample: lane l draws leg l & 1 of pair 16 unit + l / 2, row
            //    m = 2 p + leg (groups are contiguous: group g starts at row 2 g P)
            const int pairs = R.G * R.P;
            const int p0 = unit * kQPairs;
            const int p = p0 + (lane >> 1);
            if (p < pairs) {
                const int g = p / R.P;
                sample_leg(R.sa, R.groups[g], R.lobes, p - g * R.P, lane & 1);
            }
            __syncwarp();
            // 2. render the unit's perturbations, one after another by the whole warp
            const int rows = 2 * min(kQPairs, pairs - p0);
            for (int q = 0; q < rows; ++q) {
                const int m = 2 * p0 + q;
                const float* t = R.sa.tau + (size_t)m * R.n;
                float loss;
                if (kKind == HR_SCENE_DISC2D) {
                    const float cx = __fadd_rn(R.theta32[0], t[0]);
                    const float cy = __fadd_rn(R.theta32[1], t[1]);
                    loss = disc_loss_warp(A.target, A.tb, A.W, A.H, A.radius, s_px, s_py, cx, cy, lane);
                } else {
                    if (lane < R.n) s_c[warp][lane] = __fadd_rn(R.theta32[lane], t[lane]);
                    __syncwarp();
                    loss = boxes_loss_warp(A.target, A.tb, A.W, A.H, A.radius, s_px, s_py, s_c[warp], s_sp[warp],
                                           R.n / 2, lane);
                    __syncwarp();
                }
                if (lane == 0) R.loss[m] = loss;
            }
            // 3. count the unit (weights and losses visible GPU-wide first); the
            //    warp that finishes the request forms its sums
            __threadfence();
            __syncwarp();
            unsigned prev = 0;
            if (lane == 0) {
                prev = atomicAdd(R.done, 1u);
                __threadfence();
            }
            __syncwarp();
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev + 1 == (unsigned)R.units) {
                queue_finalize(R, lane);
                if (lane == 0) {
                    *reinterpret_cast<volatile unsigned*>(R.done) = 0u;
                    __threadfence_system();
                    st_release_sys(R.flag, 1);
                }
            }
            __syncwarp();
            // the next unit: wait for it unless its descriptor is already coming
            if (ready <= 0) {
                got = ticket_wait(A, lane, un, true);
                if (got > 0) unit_n = fetch_desc(A, lane, un, &s_req[warp][1 - cur]);
            }
            cur = 1 - cur;
            unit = unit_n;
        }
        if (got < 0) code = HR_ERR_TIMEOUT;
    }
    // the last warp to leave rewinds the claim counter and records why the
    // launch ended
    if (lane == 0) {
        if (code != HR_OK) atomicCAS(&A.ctl->code, 0, code);
        __threadfence();
        if (atomicSub(&A.ctl->running, 1) == 1) {
            __threadfence();
            *reinterpret_cast<volatile unsigned long long*>(&A.ctl->claim) = ld_acquire_gpu(&A.ctl->units);
            const int c = ld_volatile(&A.ctl->code);
            __threadfence_system();
            st_release_sys(&A.host->status, c);
        }
    }
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace hr

using namespace hr;

struct hr_queue_s {
    hr_scene scene = nullptr;
    std::mutex mu;
    cudaStream_t kstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool launched = false;
    int cap = 0, grid = 0;
    long long budget = 0, safety = 0;
    uint64_t launches = 0;
    // device memory
    QCtl* ctl = nullptr;
    QReq* d_ring = nullptr;
    unsigned long long* unit_ring = nullptr;
    unsigned* done = nullptr;
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0, head = 0;
    // host-mapped memory and its device views
    QHost* host = nullptr;
    QReq* h_ring = nullptr;
    double* h_res = nullptr;
    int* h_flag = nullptr;
    QHost* dv_host = nullptr;
    QReq* dv_ring = nullptr;
    double* dv_res = nullptr;
    int* dv_flag = nullptr;
    int* h_init = nullptr;             // pinned {running, stop, code} copied at each launch
    // host bookkeeping
    uint64_t next = 0;                 // next ticket
    uint64_t units_next = 0;           // units submitted so far
    struct Inflight { uint64_t ticket; size_t start; uint64_t first_unit; };
    std::deque<Inflight> inflight;     // unfinished requests in submission order (arena owners)
    std::vector<uint64_t> slot_ticket; // ticket + 1 of the request holding each slot, 0 when free
    std::vector<int> slot_count;       // doubles of its result
};

namespace {

bool slot_finished(const hr_queue_s* q, int slot) {
    return __atomic_load_n(q->h_flag + slot, __ATOMIC_ACQUIRE) != 0;
}

// A request has finished when its flag is set, or when its slot no longer
// carries its ticket (its result was read and the slot may hold a newer one).
bool request_finished(const hr_queue_s* q, uint64_t ticket) {
    const int slot = (int)(ticket % (uint64_t)q->cap);
    return q->slot_ticket[slot] != ticket + 1 || slot_finished(q, slot);
}

// Arena blocks come back in submission order, as requests finish.
void retire(hr_queue_s* q) {
    while (!q->inflight.empty() && request_finished(q, q->inflight.front().ticket)) q->inflight.pop_front();
    if (q->inflight.empty()) q->head = 0;
}

// Start of a free arena block of `bytes`, or SIZE_MAX.  The arena is a ring:
// blocks are taken at head and freed from the oldest unfinished request's start.
size_t arena_fit(const hr_queue_s* q, size_t bytes) {
    if (q->inflight.empty()) return bytes <= q->arena_bytes ? 0 : SIZE_MAX;
    const size_t tail = q->inflight.front().start;
    if (q->head > tail) {
        if (q->head + bytes <= q->arena_bytes) return q->head;
        return bytes < tail ? 0 : SIZE_MAX;
    }
    if (q->head < tail && q->head + bytes < tail) return q->head;
    return SIZE_MAX;
}

// Launches the kernel unless one is running.  The status word is 1 from the
// launch until the kernel's last warp leaves.
hr_status ensure_running(hr_queue_s* q) {
    if (q->launched) {
        if (__atomic_load_n(&q->host->status, __ATOMIC_ACQUIRE) == 1) return HR_OK;
        const cudaError_t e = cudaEventSynchronize(q->kdone);
        if (e != cudaSuccess) return fail(HR_ERR_CUDA, "queue kernel: %s", cudaGetErrorString(e));
        q->launched = false;
    }
    const DevScene& sc = q->scene->sc;
    q->h_init[0] = q->grid * kQWarps;   // running
    q->h_init[1] = 0;                   // stop
    q->h_init[2] = 0;                   // code
    cudaError_t e = cudaMemcpyAsync(&q->ctl->running, q->h_init, 3 * sizeof(int), cudaMemcpyHostToDevice, q->kstream);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "queue launch: %s", cudaGetErrorString(e));
    __atomic_store_n(&q->host->status, 1, __ATOMIC_RELEASE);
    QArgs a{};
    a.ctl = q->ctl;
    a.host = q->dv_host;
    a.h_ring = q->dv_ring;
    a.d_ring = q->d_ring;
    a.unit_ring = q->unit_ring;
    a.cap = q->cap;
    a.W = sc.W;
    a.H = sc.H;
    a.radius = sc.radius;
    a.target = sc.target;
    a.tb = DiscBits{sc.tbinary ? sc.tbits : nullptr, sc.trowpop};
    a.budget = q->budget;
    a.safety = q->safety;
    if (q->scene->sc.kind == HR_SCENE_DISC2D) queue_kernel<HR_SCENE_DISC2D><<<q->grid, 32 * kQWarps, 0, q->kstream>>>(a);
    else queue_kernel<HR_SCENE_BOXES2D><<<q->grid, 32 * kQWarps, 0, q->kstream>>>(a);
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaEventRecord(q->kdone, q->kstream);
    if (e != cudaSuccess) {
        __atomic_store_n(&q->host->status, (int)HR_ERR_CUDA, __ATOMIC_RELEASE);
        return fail(HR_ERR_CUDA, "queue launch: %s", cudaGetErrorString(e));
    }
    q->launched = true;
    ++q->launches;
    return HR_OK;
}

void free_queue(hr_queue_s* q) {
    cudaFree(q->ctl);
    cudaFree(q->d_ring);
    cudaFree(q->unit_ring);
    cudaFree(q->done);
    cudaFree(q->arena);
    if (q->host) cudaFreeHost(q->host);
    if (q->h_ring) cudaFreeHost(q->h_ring);
    if (q->h_res) cudaFreeHost(q->h_res);
    if (q->h_flag) cudaFreeHost(q->h_flag);
    if (q->h_init) cudaFreeHost(q->h_init);
    if (q->kdone) cudaEventDestroy(q->kdone);
    if (q->kstream) cudaStreamDestroy(q->kstream);
    delete q;
}

// Checks one request and writes its descriptor into the host ring; the
// caller holds the queue lock, has checked the options, and publishes.
hr_status queue_push(hr_queue_s* q, int32_t quantity, const double* h_theta, const double* h_v, const hr_opts* o,
                     uint64_t* ticket) {
    const int n = q->scene->sc.n;
    const int E = n_elements(quantity, n);
    const int G = o->strategy == HR_ELEMENTWISE ? E : 1;
    if (n > kQMaxN || G > kQMaxGroups)
        return fail(HR_ERR_UNSUPPORTED, "queued requests have at most %d groups", kQMaxGroups);
    const int P = (int)(o->n_perturb / 2);
    const int64_t Mt = (int64_t)G * o->n_perturb;
    const size_t bytes = up256(sizeof(float) * Mt * n) + up256(sizeof(float) * Mt * E) + up256(sizeof(float) * Mt);
    if (bytes > q->arena_bytes)
        return fail(HR_ERR_INVALID_ARG, "the request needs %zu bytes, more than the arena", bytes);
    const int units = (G * P + kQPairs - 1) / kQPairs;
    if (units > kQUnitRing) return fail(HR_ERR_INVALID_ARG, "more than %d units of %d pairs", kQUnitRing, kQPairs);
    retire(q);
    const int slot = (int)(q->next % (uint64_t)q->cap);
    if (q->slot_ticket[slot] != 0)
        return fail(HR_ERR_BUSY, "ring full: ticket %llu not yet waited for",
                    (unsigned long long)(q->slot_ticket[slot] - 1));
    const size_t start = arena_fit(q, bytes);
    if (start == SIZE_MAX) return fail(HR_ERR_BUSY, "arena full");
    // a unit ring entry is rewritten kQUnitRing units later: every unit from the
    // oldest unfinished request's first to this request's last must fit
    if (!q->inflight.empty() && q->units_next + units - q->inflight.front().first_unit > (uint64_t)kQUnitRing)
        return fail(HR_ERR_BUSY, "unit ring full");
    unsigned char* base = q->arena + start;
    // the descriptor, written in place in the host ring
    QReq& R = q->h_ring[slot];
    memset(&R, 0, sizeof(R));
    R.n = n;
    R.E = E;
    R.G = G;
    R.P = P;
    R.elementwise = o->strategy == HR_ELEMENTWISE;
    R.hessian = quantity == HR_HESSIAN;
    R.inv2P = 1.0 / (double)o->n_perturb;
    R.units = units;
    for (int i = 0; i < n; ++i) R.theta32[i] = (float)h_theta[i];
    if (quantity == HR_HVP)
        for (int i = 0; i < n; ++i) R.vv[i] = h_v[i];
    R.sa.n = n;
    R.sa.E = E;
    R.sa.seed = o->seed;
    // the lobe constants as the estimate path forms them
    const double s2 = o->sigma * o->sigma;
    const double Zg = std::sqrt(2.0 / M_PI) / o->sigma;
    const double Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * s2);
    R.sa.tau = reinterpret_cast<float*>(base);
    R.sa.w = reinterpret_cast<float*>(base + up256(sizeof(float) * Mt * n));
    R.loss = reinterpret_cast<float*>(base + up256(sizeof(float) * Mt * n) + up256(sizeof(float) * Mt * E));
    R.lobes = make_lobes(o->sigma, Zg, Zd, Zg * Zg, n);
    for (int g = 0; g < G; ++g) {
        SampleGroup& gr = R.groups[g];
        gr.m0 = (int32_t)(g * o->n_perturb);
        gr.P = P;
        gr.lobe = quantity == HR_GRAD ? 0 : 1;
        gr.quantity = quantity;
        gr.sub = o->sub + (uint32_t)g;
        gr.request = o->request_id;
        if (o->strategy == HR_AGGREGATE) {
            gr.comp_i = -1; gr.comp_j = -1;
        } else if (o->strategy == HR_PLAIN) {
            gr.comp_i = -3; gr.comp_j = -3;
        } else if (quantity == HR_GRAD) {
            gr.comp_i = g; gr.comp_j = g;
        } else if (quantity == HR_HVP) {
            gr.comp_i = g; gr.comp_j = -2; gr.quantity = 4;   // row g of the HVP, row-mixture draws
        } else {
            int r = 0, rem = g;
            while (rem >= n - r) { rem -= n - r; ++r; }
            gr.comp_i = r; gr.comp_j = r + rem;
        }
    }
    R.res = q->dv_res + (size_t)slot * kQMaxResult;
    R.flag = q->dv_flag + slot;
    R.done = q->done + slot;
    q->h_flag[slot] = 0;
    q->slot_ticket[slot] = q->next + 1;
    q->slot_count[slot] = quantity == HR_HESSIAN ? n * n : n;
    q->inflight.push_back({q->next, start, q->units_next});
    q->units_next += (uint64_t)units;
    q->head = start + bytes;
    *ticket = q->next++;
    return HR_OK;
}

// Checks of one request that need no queue state.
hr_status queue_check(hr_queue_s* q, int32_t quantity, const double* h_theta, const double* h_v, const hr_opts* o) {
    if (!h_theta || !o) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    if (quantity != HR_GRAD && quantity != HR_HESSIAN && quantity != HR_HVP)
        return fail(HR_ERR_INVALID_ARG, "unknown quantity %d", quantity);
    if (quantity == HR_HVP && !h_v) return fail(HR_ERR_INVALID_ARG, "an HVP needs v");
    return validate_opts(q->scene, quantity, o);
}

void queue_publish(hr_queue_s* q) {
    // the descriptors' stores come before the count (release)
    __atomic_store_n(&q->host->submitted, (unsigned long long)q->next, __ATOMIC_RELEASE);
}

}  // namespace

extern "C" {

hr_status hr_queue_create(hr_scene scene, const hr_queue_opts* o, hr_queue* out) {
    clear_error();
    if (!scene || !o || !out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (scene->sc.kind != HR_SCENE_DISC2D && scene->sc.kind != HR_SCENE_BOXES2D)
        return fail(HR_ERR_UNSUPPORTED, "the persistent queue serves disc and squares scenes");
    if (scene->sc.n > kQMaxN) return fail(HR_ERR_UNSUPPORTED, "queued scenes have at most %d parameters", kQMaxN);
    if (o->max_requests < 1 || o->max_requests > 16384)
        return fail(HR_ERR_INVALID_ARG, "max_requests must be 1..16384");
    if (o->arena_bytes < (1 << 20)) return fail(HR_ERR_INVALID_ARG, "arena_bytes must be at least 1 MiB");
    if (o->idle_budget_us < 1 || o->idle_budget_us > 10000000)
        return fail(HR_ERR_INVALID_ARG, "idle_budget_us must be 1..10^7");
    hr_queue_s* q = new hr_queue_s();
    q->scene = scene;
    q->cap = o->max_requests;
    q->arena_bytes = (size_t)o->arena_bytes;
    int dev = 0, clock_khz = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    auto step = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    step(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
    step(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (scene->sc.kind == HR_SCENE_DISC2D)
        step(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel<HR_SCENE_DISC2D>, 32 * kQWarps, 0));
    else
        step(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel<HR_SCENE_BOXES2D>, 32 * kQWarps, 0));
    q->grid = sms * std::max(per_sm, 1);
    // clock64() counts SM cycles; the budget is converted at the maximum clock
    // (a lower clock only makes the wall-clock wait longer)
    const long long khz = clock_khz > 0 ? clock_khz : 2070000;
    q->budget = (long long)o->idle_budget_us * khz / 1000;
    q->safety = 4 * q->budget + 200LL * khz;   // the budget x 4 + 200 ms
    step(cudaStreamCreateWithFlags(&q->kstream, cudaStreamNonBlocking));
    step(cudaEventCreateWithFlags(&q->kdone, cudaEventDisableTiming));
    step(cudaMalloc((void**)&q->ctl, sizeof(QCtl)));
    step(cudaMemset(q->ctl, 0, sizeof(QCtl)));
    step(cudaMalloc((void**)&q->d_ring, sizeof(QReq) * kQReplicas * q->cap));
    step(cudaMalloc((void**)&q->unit_ring, sizeof(unsigned long long) * kQUnitRing));
    step(cudaMalloc((void**)&q->done, sizeof(unsigned) * q->cap));
    step(cudaMemset(q->done, 0, sizeof(unsigned) * q->cap));
    step(cudaMalloc((void**)&q->arena, q->arena_bytes));
    step(cudaHostAlloc((void**)&q->host, sizeof(QHost), cudaHostAllocMapped));
    step(cudaHostAlloc((void**)&q->h_ring, sizeof(QReq) * q->cap, cudaHostAllocMapped));
    step(cudaHostAlloc((void**)&q->h_res, sizeof(double) * kQMaxResult * q->cap, cudaHostAllocMapped));
    step(cudaHostAlloc((void**)&q->h_flag, sizeof(int) * q->cap, cudaHostAllocMapped));
    step(cudaHostAlloc((void**)&q->h_init, 4 * sizeof(int), cudaHostAllocDefault));
    if (e == cudaSuccess) {
        step(cudaHostGetDevicePointer((void**)&q->dv_host, q->host, 0));
        step(cudaHostGetDevicePointer((void**)&q->dv_ring, q->h_ring, 0));
        step(cudaHostGetDevicePointer((void**)&q->dv_res, q->h_res, 0));
        step(cudaHostGetDevicePointer((void**)&q->dv_flag, q->h_flag, 0));
    }
    step(cudaDeviceSynchronize());
    if (e != cudaSuccess) {
        free_queue(q);
        return fail(HR_ERR_OOM, "queue: %s", cudaGetErrorString(e));
    }
    memset(q->host, 0, sizeof(QHost));
    memset(q->h_flag, 0, sizeof(int) * q->cap);
    q->slot_ticket.assign(q->cap, 0);
    q->slot_count.assign(q->cap, 0);
    *out = q;
    return HR_OK;
}

hr_status hr_queue_submit(hr_queue q, int32_t quantity, const double* h_theta, const double* h_v, const hr_opts* o,
                          uint64_t* ticket) {
    clear_error();
    if (!q || !ticket) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    hr_status st;
    {
        std::lock_guard<std::mutex> lk2(q->scene->mu);
        st = queue_check(q, quantity, h_theta, h_v, o);
    }
    if (st == HR_OK) st = queue_push(q, quantity, h_theta, h_v, o, ticket);
    if (st != HR_OK) return st;
    queue_publish(q);
    return ensure_running(q);
}

hr_status hr_queue_submit_many(hr_queue q, int32_t count, int32_t quantity, const double* h_theta, const double* h_v,
                               const hr_opts* opts, uint64_t* tickets, int32_t* submitted) {
    clear_error();
    if (!q || !tickets || !submitted || !opts || count < 0) return fail(HR_ERR_INVALID_ARG, "NULL argument or count < 0");
    *submitted = 0;
    if (count == 0) return HR_OK;
    if (!h_theta) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    const int n = q->scene->sc.n;
    hr_status st = HR_OK;
    {
        std::lock_guard<std::mutex> lk2(q->scene->mu);
        for (int i = 0; i < count && st == HR_OK; ++i)
            st = queue_check(q, quantity, h_theta + (size_t)i * n, h_v ? h_v + (size_t)i * n : nullptr, opts + i);
    }
    if (st != HR_OK) return st;
    int k = 0;
    for (; k < count; ++k) {
        st = queue_push(q, quantity, h_theta + (size_t)k * n, h_v ? h_v + (size_t)k * n : nullptr, opts + k,
                        tickets + k);
        if (st != HR_OK) break;
    }
    *submitted = k;
    if (k > 0) {
        queue_publish(q);
        const hr_status rs = ensure_running(q);
        if (rs != HR_OK) return rs;
    }
    return st;
}

hr_status hr_queue_wait(hr_queue q, uint64_t ticket, double* h_out, int32_t timeout_ms) {
    clear_error();
    if (!q || !h_out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    const auto t0 = std::chrono::steady_clock::now();
    for (int spin = 0;; ++spin) {
        {
            std::lock_guard<std::mutex> lk(q->mu);
            const int slot = (int)(ticket % (uint64_t)q->cap);
            if (ticket >= q->next || q->slot_ticket[slot] != ticket + 1)
                return fail(HR_ERR_INVALID_ARG, "unknown ticket or already waited for");
            if (slot_finished(q, slot)) {
                memcpy(h_out, q->h_res + (size_t)slot * kQMaxResult, sizeof(double) * q->slot_count[slot]);
                q->slot_ticket[slot] = 0;
                retire(q);
                return HR_OK;
            }
            const hr_status rs = ensure_running(q);
            if (rs != HR_OK) return rs;
        }
        if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return fail(HR_ERR_TIMEOUT, "request not finished within %d ms", timeout_ms);
        if (spin > 1000) std::this_thread::sleep_for(std::chrono::microseconds(20));
        else std::this_thread::yield();
    }
}

hr_status hr_queue_wait_many(hr_queue q, int32_t count, const uint64_t* tickets, double* h_out, int32_t out_stride,
                             int32_t timeout_ms) {
    clear_error();
    if (!q || (count > 0 && (!tickets || !h_out)) || count < 0) return fail(HR_ERR_INVALID_ARG, "NULL argument or count < 0");
    {
        std::lock_guard<std::mutex> lk(q->mu);
        for (int i = 0; i < count; ++i) {
            const int slot = (int)(tickets[i] % (uint64_t)q->cap);
            if (tickets[i] >= q->next || q->slot_ticket[slot] != tickets[i] + 1)
                return fail(HR_ERR_INVALID_ARG, "unknown ticket %llu or already waited for",
                            (unsigned long long)tickets[i]);
            if (q->slot_count[slot] > out_stride)
                return fail(HR_ERR_INVALID_ARG, "out_stride %d below a result's %d doubles", out_stride,
                            q->slot_count[slot]);
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < count; ++i) {
        int32_t left = timeout_ms;
        if (timeout_ms >= 0) {
            const auto used = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
            left = (int32_t)std::max<long long>(0, timeout_ms - (long long)used.count());
        }
        const hr_status st = hr_queue_wait(q, tickets[i], h_out + (size_t)i * out_stride, left);
        if (st != HR_OK) return st;
    }
    return HR_OK;
}

hr_status hr_queue_status(hr_queue q, int32_t* kernel_status, uint64_t* launches) {
    clear_error();
    if (!q || !kernel_status) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    *kernel_status = __atomic_load_n(&q->host->status, __ATOMIC_ACQUIRE);
    if (launches) *launches = q->launches;
    return HR_OK;
}

hr_status hr_queue_destroy(hr_queue q) {
    if (!q) return HR_OK;
    hr_status st = HR_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (q->launched) {
            // the dispatcher leaves once it sees stop; the workers leave once the
            // device ring is empty
            __atomic_store_n(&q->host->stop, 1, __ATOMIC_RELEASE);
            const cudaError_t e = cudaEventSynchronize(q->kdone);
            if (e != cudaSuccess) st = fail(HR_ERR_CUDA, "queue kernel: %s", cudaGetErrorString(e));
        }
    }
    free_queue(q);
    return st;
}

}  // extern "C"
