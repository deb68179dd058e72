// batch.cu -- many independent reconstructions as one unit of work (the batched form
// of Section 3.4's steps 1-4): worker streams, one persistent spreading launch per
// channel over all plans, capture into a CUDA graph, and a tuner for the stream count
// and the spreading work-item size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "firm_internal.h"

using namespace firm;

struct firm_batch_s {
    int n = 0;
    std::vector<firm_plan_s*> plans;
    std::vector<int> order;                 // plans by estimated cost, largest first
    int W = 6;
    KbPoly poly{};
    int num_sms = 0;
    cudaStream_t user = nullptr;            // the caller's stream
    cudaStream_t main = nullptr;            // the batch's own (capturable) stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_fork, ev_join;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
    int n_streams = 1;                      // active worker streams
    int chunk = kChunk;
    // device workspace (caller's)
    char* desc_k = nullptr;                 // n spreading descriptors, kernel channel
    char* desc_r = nullptr;                 // n spreading descriptors, A*b channel
    int* item_off = nullptr;                // 2 x (n + 1)
    int* queue = nullptr;                   // 2
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<firm_batch_item> cap_items;
    int cap_iters = -1, cap_flags = -1, cap_streams = -1, cap_chunk = -1;
    double cap_tol = -1.0;
    long long launches_per_run = 0;
    int last_iters = 0;
    bool ran = false;
    // firm_batch_solve: the learned network (caller's device buffers), its per-plan inputs
    // and tables, the MLP scratch, the plans' CG states and the count of plans not done
    const void* net_bf16 = nullptr;
    const float* net = nullptr;
    float* feat = nullptr;                  // n x 1024 network inputs
    float* tab = nullptr;                   // n x 1024 network outputs (log tables)
    float* mlp_work = nullptr;
    CgState** cg_ptrs = nullptr;            // n device pointers
    int* not_done = nullptr;                // n ints: 1 while plan i has not stopped
    cudaGraph_t cg_graph = nullptr;         // one chunk of CG iterations of every plan
    cudaGraphExec_t cg_exec = nullptr;
    int cg_cap_streams = -1;
    std::vector<char> cg_cap_pc;            // use_pc of every plan when the chunk was captured
    std::vector<int> cg_cap_active;         // the plans the captured chunk iterates
    std::vector<int> cap_pc_modes;          // the plans' preconditioner modes at the front's capture
    std::vector<char> cap_use_pc;           // use_pc the captured front sets
    std::vector<char> use_pc;               // per plan: preconditioned CG in the current solve
    double last_tol = 0.0;                  // rel_tol of the last run (0: fixed iterations)
};

namespace {

// The descriptors form a plain device array (the kernel indexes it by element), so
// their host packing uses the element size itself.
size_t desc_stride() { return spread_batch_desc_bytes(); }

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// [descriptors, kernel channel | descriptors, A*b channel | item offsets | queues |
//  network inputs | network outputs | MLP scratch | CG state pointers | not-done count]
size_t desc_region(int n) { return round256(desc_stride() * (size_t)n); }
size_t off_region(int n) { return round256(2 * (size_t)(n + 1) * sizeof(int)); }
size_t net_region(int n) { return round256((size_t)n * 1024 * sizeof(float)); }
size_t mlp_region(int n) { return round256(firm_mlp_work_floats(n) * sizeof(float)); }
size_t ptr_region(int n) { return round256((size_t)n * sizeof(CgState*)); }
size_t flag_region(int n) { return round256((size_t)n * sizeof(int)); }
size_t batch_bytes(int n) {
    return 2 * desc_region(n) + off_region(n) + 256 + 2 * net_region(n) + mlp_region(n) + ptr_region(n) +
           flag_region(n);
}

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool same_items(const std::vector<firm_batch_item>& a, const firm_batch_item* b, int n) {
    if ((int)a.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (a[i].M != b[i].M || a[i].R != b[i].R || a[i].group != b[i].group || a[i].images != b[i].images ||
            a[i].shifts != b[i].shifts || a[i].x != b[i].x)
            return false;
    return true;
}

#define BCK(x)                                    \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

// Everything up to (not including) the kernel-channel spreading, for one plan.
cudaError_t plan_front(Plan& P, const firm_batch_item& it, bool spread_here) {
    Workspace& w = P.ws;
    const int M = it.M;
    P.cur_R = it.R;
    P.cur_images = it.images;
    if (it.group) P.cur_gid = it.group;
    else { BCK(cudaMemsetAsync(w.gid, 0, sizeof(int32_t) * (M > 0 ? M : 1), P.stream)); P.cur_gid = w.gid; }
    if (it.shifts) P.cur_shifts = it.shifts;
    else { BCK(cudaMemsetAsync(w.shifts, 0, sizeof(double) * 2 * (M > 0 ? M : 1), P.stream)); P.cur_shifts = w.shifts; }
    BCK(cudaMemsetAsync(w.counters + 2, 0, sizeof(int), P.stream));
    BCK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += M > 0 ? 1 : 0;
    BCK(launch_bin(P, M, true));
    BCK(launch_spread_clear(P, true));
    if (spread_here) BCK(launch_spread_only(P, M, true));
    P.last_M = M;
    if (M > 0) BCK(launch_view_axis(P, P.cur_R, M));     // the preconditioners' cone axis
    return cudaSuccess;
}

// Ker transform, K-hat, lam_eff, image DFT and A*b binning (spreading after it).
cudaError_t plan_middle(Plan& P, const firm_batch_item& it, bool spread_here) {
    const int M = it.M;
    BCK(launch_ker_transform(P));
    BCK(launch_khat(P));
    BCK(launch_lam_eff(P));
    BCK(launch_damping(P));
    BCK(launch_image_dft(P, M, P.cur_images, P.cur_shifts, P.cur_gid));
    BCK(launch_bin(P, M, false));
    BCK(launch_spread_clear(P, false));
    if (spread_here) BCK(launch_spread_only(P, M, false));
    return cudaSuccess;
}

// A*b transform, then `iters` CG iterations from x0 = 0 (no tolerance), volume out.
cudaError_t plan_back(Plan& P, const firm_batch_item& it, int iters) {
    Workspace& w = P.ws;
    BCK(launch_rhs_transform(P));
    BCK(launch_cg_init(P, w.rhs, iters, 0.0, false));
    for (int k = 0; k < iters; ++k) {
        BCK(launch_toeplitz(P, w.p, w.q, w.r, w.cg, nullptr));
        BCK(launch_cg_update(P));
    }
    const size_t n3 = (size_t)P.N * P.N * P.N;
    BCK(cudaMemcpyAsync(it.x, w.x, n3 * sizeof(float), cudaMemcpyDeviceToDevice, P.stream));
    return cudaSuccess;
}

// The preconditioned solve's set-up for one plan (after its A*b transform): the
// plan's own preconditioner (or, with the batch network, the table row it produced),
// then CG initialisation from x0 = 0 with the tolerance.
cudaError_t plan_solve_init(firm_batch_s& b, int i, int max_iter, double rel_tol, bool learned) {
    Plan& P = b.plans[i]->P;
    Workspace& w = P.ws;
    bool pc = true;
    if (learned) {
        BCK(launch_pc_from_table(P, b.tab + (size_t)i * 1024));
    } else if (P.pc_mode == FIRM_PRECOND_CIRCULANT) {
        BCK(launch_chan_spectrum(P));
        BCK(launch_pc_build_circulant(P));
    } else if (P.pc_mode == FIRM_PRECOND_TABLE) {
        BCK(launch_pc_from_table(P, w.pc_table));
    } else {
        pc = false;
    }
    b.use_pc[i] = pc ? 1 : 0;
    BCK(launch_cg_init(P, w.rhs, max_iter, rel_tol, pc));
    if (pc) BCK(launch_precond(P, w.r, w.z, w.cg));
    return cudaSuccess;
}

// `its` CG iterations of one plan (kernels of a finished solve return at once).
cudaError_t plan_cg_chunk(firm_batch_s& b, int i, int its) {
    Plan& P = b.plans[i]->P;
    Workspace& w = P.ws;
    const bool pc = b.use_pc[i] != 0;
    for (int k = 0; k < its; ++k) {
        BCK(launch_toeplitz(P, w.p, w.q, w.r, w.cg, pc ? w.z : nullptr));
        BCK(launch_cg_update(P));
        if (pc) BCK(launch_precond(P, w.r, w.z, w.cg));
    }
    return cudaSuccess;
}

__global__ void k_batch_not_done(CgState* const* __restrict__ cgs, int n, int* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = cgs[i]->done ? 0 : 1;
}

cudaError_t fork(firm_batch_s& b) {
    BCK(cudaEventRecord(b.ev_fork[0], b.main));
    for (int s = 0; s < b.n_streams; ++s) BCK(cudaStreamWaitEvent(b.streams[s], b.ev_fork[0], 0));
    return cudaSuccess;
}

cudaError_t join(firm_batch_s& b) {
    for (int s = 0; s < b.n_streams; ++s) {
        BCK(cudaEventRecord(b.ev_join[s], b.streams[s]));
        BCK(cudaStreamWaitEvent(b.main, b.ev_join[s], 0));
    }
    return cudaSuccess;
}

// The whole batch in stream order on b.main (and the worker streams forked from it).
cudaError_t enqueue_body(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol);

cudaError_t enqueue(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol) {
    std::vector<cudaStream_t> saved(b.n);
    for (int i = 0; i < b.n; ++i) saved[i] = b.plans[i]->P.stream;
    const cudaError_t e = enqueue_body(b, items, iters, flags, rel_tol);
    for (int i = 0; i < b.n; ++i) b.plans[i]->P.stream = saved[i];
    return e;
}

// Flag bit of an enqueue for firm_batch_solve (not a public flag): the front of the
// batch up to the CG set-up; the iterations then run in chunks.
constexpr int kSolveFront = 1 << 16;
cudaError_t enqueue_body(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol) {
    const bool persistent = (flags & FIRM_BATCH_PERSISTENT) != 0;
    const bool solve = (flags & kSolveFront) != 0;
    const bool learned = solve && (flags & FIRM_BATCH_LEARNED) != 0;
    long long l0 = 0;
    for (auto* h : b.plans) l0 += h->P.launches;
    long long own = 0;
    BCK(fork(b));
    for (int k = 0; k < b.n; ++k) {
        const int i = b.order[k];
        Plan& P = b.plans[i]->P;
        P.stream = b.streams[k % b.n_streams];
        BCK(plan_front(P, items[i], !persistent));
        if (!persistent) BCK(plan_middle(P, items[i], true));
    }
    if (persistent) {
        BCK(join(b));
        BCK(launch_spread_batch(b.n, true, b.W, b.poly, b.desc_k, b.item_off, b.queue, b.num_sms, b.main));
        own += 2;
        BCK(fork(b));
        for (int k = 0; k < b.n; ++k) {
            const int i = b.order[k];
            BCK(plan_middle(b.plans[i]->P, items[i], false));
        }
        BCK(join(b));
        BCK(launch_spread_batch(b.n, false, b.W, b.poly, b.desc_r, b.item_off + b.n + 1, b.queue + 1, b.num_sms,
                                b.main));
        own += 2;
        BCK(fork(b));
    }
    if (!solve) {
        for (int k = 0; k < b.n; ++k) {
            const int i = b.order[k];
            BCK(plan_back(b.plans[i]->P, items[i], iters));
        }
    } else {
        for (int k = 0; k < b.n; ++k) {
            const int i = b.order[k];
            Plan& P = b.plans[i]->P;
            BCK(launch_rhs_transform(P));
            if (learned) {
                // the network input of this plan's kernel, row i of the batch's inputs
                BCK(launch_pc_features(P, items[i].M, P.ws.pc_feat));
                BCK(launch_pc_normalize(P, P.ws.pc_feat, b.feat + (size_t)i * 1024));
            }
        }
        if (learned) {
            // one forward pass of the network over every plan's input (BF16 weights)
            BCK(join(b));
            if (firm_mlp_forward_bf16(b.net_bf16, b.net, b.n, b.feat, b.tab, b.mlp_work, b.main) != FIRM_OK)
                return cudaErrorUnknown;
            own += 3;
            BCK(fork(b));
        }
        for (int k = 0; k < b.n; ++k) BCK(plan_solve_init(b, b.order[k], iters, rel_tol, learned));
    }
    BCK(join(b));
    long long l1 = 0;
    for (auto* h : b.plans) l1 += h->P.launches;
    b.launches_per_run = l1 - l0 + own;
    return cudaSuccess;
}

// Spreading descriptors depend on the items' group pointers (and on nothing that a
// batch run changes otherwise); written before the run or the capture.
cudaError_t write_desc(firm_batch_s& b, const firm_batch_item* items) {
    const size_t st = desc_stride();
    std::vector<char> hk(st * b.n), hr(st * b.n);
    for (int i = 0; i < b.n; ++i) {
        Plan& P = b.plans[i]->P;
        P.cur_gid = items[i].group ? items[i].group : P.ws.gid;
        spread_batch_fill_desc(P, true, hk.data() + st * i);
        spread_batch_fill_desc(P, false, hr.data() + st * i);
    }
    BCK(cudaMemcpyAsync(b.desc_k, hk.data(), hk.size(), cudaMemcpyHostToDevice, b.main));
    BCK(cudaMemcpyAsync(b.desc_r, hr.data(), hr.size(), cudaMemcpyHostToDevice, b.main));
    return cudaStreamSynchronize(b.main);
}

void drop_graph(firm_batch_s& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
    b.cap_items.clear();
    b.cap_iters = b.cap_flags = b.cap_streams = b.cap_chunk = -1;
    b.cap_tol = -1.0;
}

void drop_cg_graph(firm_batch_s& b) {
    if (b.cg_exec) cudaGraphExecDestroy(b.cg_exec);
    if (b.cg_graph) cudaGraphDestroy(b.cg_graph);
    b.cg_exec = nullptr;
    b.cg_graph = nullptr;
    b.cg_cap_streams = -1;
    b.cg_cap_pc.clear();
    b.cg_cap_active.clear();
}

constexpr int kCgChunk = 8;      // CG iterations per plan between two reads of the stop count

// One chunk of CG iterations of the plans in `active` (largest first) on the worker
// streams, then every plan's not-stopped flag into b.not_done (queued on b.main).
cudaError_t enqueue_cg_chunk(firm_batch_s& b, const std::vector<int>& active) {
    std::vector<cudaStream_t> saved(b.n);
    for (int i = 0; i < b.n; ++i) saved[i] = b.plans[i]->P.stream;
    cudaError_t e = fork(b);
    for (size_t k = 0; k < active.size() && e == cudaSuccess; ++k) {
        const int i = active[k];
        b.plans[i]->P.stream = b.streams[k % b.n_streams];
        e = plan_cg_chunk(b, i, kCgChunk);
    }
    if (e == cudaSuccess) e = join(b);
    if (e == cudaSuccess) {
        k_batch_not_done<<<(b.n + 255) / 256, 256, 0, b.main>>>(b.cg_ptrs, b.n, b.not_done);
        e = cudaGetLastError();
    }
    for (int i = 0; i < b.n; ++i) b.plans[i]->P.stream = saved[i];
    return e;
}

// Chunks until every plan has stopped (tolerance, max_iter or breakdown).  With `graph`
// the chunk is captured as a CUDA graph over the plans still running, and captured
// again, over fewer plans, once a quarter of those have stopped (a stopped plan's
// kernels return at once, but each launch still costs).  The host reads the plans'
// flags after each chunk.
int run_cg_chunks(firm_batch_s& b, int max_iter, bool graph) {
    std::vector<int> active;
    for (int k = 0; k < b.n; ++k) active.push_back(b.order[k]);
    std::vector<int> flags(b.n, 1);
    for (int done_its = 0; done_its < max_iter && !active.empty(); done_its += kCgChunk) {
        // the captured chunk must iterate every running plan (a plan it leaves out would
        // never move); it may hold stopped ones until a quarter of its plans have stopped
        bool covers = true;
        for (int i : active)
            covers = covers && std::find(b.cg_cap_active.begin(), b.cg_cap_active.end(), i) != b.cg_cap_active.end();
        if (graph && (!b.cg_exec || b.cg_cap_streams != b.n_streams || b.cg_cap_pc != b.use_pc || !covers ||
                      (b.cg_cap_active != active && 4 * active.size() <= 3 * b.cg_cap_active.size()))) {
            drop_cg_graph(b);
            if (cudaStreamBeginCapture(b.main, cudaStreamCaptureModeRelaxed) != cudaSuccess) return FIRM_ECUDA;
            const cudaError_t e = enqueue_cg_chunk(b, active);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(b.main, &g);
            if (e != cudaSuccess || e2 != cudaSuccess || !g) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return FIRM_ECUDA;
            }
            b.cg_graph = g;
            if (cudaGraphInstantiate(&b.cg_exec, b.cg_graph, 0) != cudaSuccess) {
                drop_cg_graph(b);
                return FIRM_ECUDA;
            }
            b.cg_cap_streams = b.n_streams;
            b.cg_cap_pc = b.use_pc;
            b.cg_cap_active = active;
        }
        if (graph) {
            if (cudaGraphLaunch(b.cg_exec, b.main) != cudaSuccess) return FIRM_ECUDA;
        } else if (enqueue_cg_chunk(b, active) != cudaSuccess) {
            return FIRM_ECUDA;
        }
        if (cudaMemcpyAsync(flags.data(), b.not_done, sizeof(int) * b.n, cudaMemcpyDeviceToHost, b.main) !=
                cudaSuccess ||
            cudaStreamSynchronize(b.main) != cudaSuccess)
            return FIRM_ECUDA;
        std::vector<int> still;
        for (int i : active)
            if (flags[i]) still.push_back(i);
        active.swap(still);
    }
    return FIRM_OK;
}

int check_items(const firm_batch_s& b, const firm_batch_item* items) {
    if (!items) return FIRM_EINVAL;
    for (int i = 0; i < b.n; ++i) {
        const firm_batch_item& it = items[i];
        const Plan& P = b.plans[i]->P;
        if (it.M < 0 || it.M > P.p.M || !it.x || !dev_ptr(it.x)) return FIRM_EINVAL;
        if (it.M > 0 && (!dev_ptr(it.R) || !dev_ptr(it.images))) return FIRM_EINVAL;
        if (it.M > 0 && (reinterpret_cast<uintptr_t>(it.images) & 15)) return FIRM_EINVAL;   // bulk-copied
        if (it.group && !dev_ptr(it.group)) return FIRM_EINVAL;
        if (it.shifts && !dev_ptr(it.shifts)) return FIRM_EINVAL;
    }
    return FIRM_OK;
}

int run_main(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol);

// The batch runs on its own stream, ordered after the caller's stream and before what
// the caller queues next on it.
int run(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol = 0.0) {
    if (cudaEventRecord(b.ev_in, b.user) != cudaSuccess || cudaStreamWaitEvent(b.main, b.ev_in, 0) != cudaSuccess)
        return FIRM_ECUDA;
    const int st = run_main(b, items, iters, flags, rel_tol);
    if (st != FIRM_OK) return st;
    if (cudaEventRecord(b.ev_out, b.main) != cudaSuccess || cudaStreamWaitEvent(b.user, b.ev_out, 0) != cudaSuccess)
        return FIRM_ECUDA;
    return FIRM_OK;
}

int run_main(firm_batch_s& b, const firm_batch_item* items, int iters, int flags, double rel_tol) {
    const bool graph = (flags & FIRM_BATCH_GRAPH) != 0;
    for (auto* h : b.plans) h->P.chunk = b.chunk;
    std::vector<int> modes(b.n);
    for (int i = 0; i < b.n; ++i) modes[i] = b.plans[i]->P.pc_mode;
    if (graph && b.exec && b.cap_iters == iters && b.cap_flags == flags && b.cap_streams == b.n_streams &&
        b.cap_chunk == b.chunk && b.cap_tol == rel_tol && b.cap_pc_modes == modes &&
        same_items(b.cap_items, items, b.n)) {
        // the replayed front set use_pc as at its capture
        if (flags & kSolveFront) b.use_pc = b.cap_use_pc;
        if (cudaGraphLaunch(b.exec, b.main) != cudaSuccess) return FIRM_ECUDA;
        b.last_iters = iters;
        b.ran = true;
        return FIRM_OK;
    }
    if (write_desc(b, items) != cudaSuccess) return FIRM_ECUDA;
    if (!graph) {
        if (enqueue(b, items, iters, flags, rel_tol) != cudaSuccess) return FIRM_ECUDA;
        b.last_iters = iters;
        b.ran = true;
        return FIRM_OK;
    }
    drop_graph(b);
    if (cudaStreamBeginCapture(b.main, cudaStreamCaptureModeRelaxed) != cudaSuccess) return FIRM_ECUDA;
    const cudaError_t e = enqueue(b, items, iters, flags, rel_tol);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b.main, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return FIRM_ECUDA;
    }
    b.graph = g;
    if (cudaGraphInstantiate(&b.exec, b.graph, 0) != cudaSuccess) {
        drop_graph(b);
        return FIRM_ECUDA;
    }
    b.cap_items.assign(items, items + b.n);
    b.cap_pc_modes = modes;
    b.cap_use_pc = b.use_pc;
    b.cap_tol = rel_tol;
    b.cap_iters = iters;
    b.cap_flags = flags;
    b.cap_streams = b.n_streams;
    b.cap_chunk = b.chunk;
    if (cudaGraphLaunch(b.exec, b.main) != cudaSuccess) return FIRM_ECUDA;
    b.last_iters = iters;
    b.ran = true;
    return FIRM_OK;
}

}  // namespace

extern "C" {

int firm_batch_workspace_size(int n_plans, size_t* bytes) {
    if (n_plans < 1 || n_plans > kMaxBatch || !bytes) return FIRM_EINVAL;
    *bytes = batch_bytes(n_plans);
    return FIRM_OK;
}

int firm_batch_create(firm_batch_t* out, int n_plans, const firm_plan_t* plans, int n_streams, void* workspace,
                      size_t workspace_bytes, void* stream) {
    if (!out) return FIRM_EINVAL;
    *out = nullptr;
    if (n_plans < 1 || n_plans > kMaxBatch || !plans || n_streams < 1 || n_streams > 64) return FIRM_EINVAL;
    if (!workspace || workspace_bytes < batch_bytes(n_plans)) return FIRM_ENOMEM;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0 || !dev_ptr(workspace)) return FIRM_EINVAL;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return FIRM_EINVAL;
        if (plans[i]->P.p.W != plans[0]->P.p.W) return FIRM_EINVAL;
        if (plans[i]->P.p.flags & FIRM_FLAG_FP64_CG) return FIRM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return FIRM_EINVAL;
    }
    firm_batch_s* b = new (std::nothrow) firm_batch_s();
    if (!b) return FIRM_ENOMEM;
    b->n = n_plans;
    b->plans.assign(plans, plans + n_plans);
    b->W = plans[0]->P.p.W;
    b->poly = plans[0]->P.poly;
    b->num_sms = plans[0]->P.num_sms;
    b->user = reinterpret_cast<cudaStream_t>(stream);
    b->n_streams = std::min(n_streams, n_plans);
    char* base = reinterpret_cast<char*>(workspace);
    b->desc_k = base;
    b->desc_r = base + desc_region(n_plans);
    b->item_off = reinterpret_cast<int*>(base + 2 * desc_region(n_plans));
    b->queue = reinterpret_cast<int*>(base + 2 * desc_region(n_plans) + off_region(n_plans));
    char* tail = base + 2 * desc_region(n_plans) + off_region(n_plans) + 256;
    b->feat = reinterpret_cast<float*>(tail);
    b->tab = reinterpret_cast<float*>(tail + net_region(n_plans));
    b->mlp_work = reinterpret_cast<float*>(tail + 2 * net_region(n_plans));
    b->cg_ptrs = reinterpret_cast<CgState**>(tail + 2 * net_region(n_plans) + mlp_region(n_plans));
    b->not_done = reinterpret_cast<int*>(tail + 2 * net_region(n_plans) + mlp_region(n_plans) + ptr_region(n_plans));
    b->use_pc.assign(n_plans, 0);
    b->streams.assign(n_streams, nullptr);
    b->ev_join.assign(n_streams, nullptr);
    b->ev_fork.assign(1, nullptr);
    bool ok = true;
    for (int s = 0; s < n_streams && ok; ++s) {
        ok = cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev_join[s], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_fork[0], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreate(&b->ev_t0) == cudaSuccess && cudaEventCreate(&b->ev_t1) == cudaSuccess;
    if (!ok) {
        firm_batch_destroy(b);
        return FIRM_ECUDA;
    }
    {
        std::vector<CgState*> cgp(n_plans);
        for (int i = 0; i < n_plans; ++i) cgp[i] = plans[i]->P.ws.cg;
        if (cudaMemcpy(b->cg_ptrs, cgp.data(), sizeof(CgState*) * n_plans, cudaMemcpyHostToDevice) != cudaSuccess) {
            firm_batch_destroy(b);
            return FIRM_ECUDA;
        }
    }
    // largest first: spreading ~ points, CG ~ iterations x (2N)^3 (order fixed at create)
    std::vector<double> cost(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        const Plan& P = plans[i]->P;
        const double n2 = 8.0 * P.N * P.N * P.N;
        cost[i] = (double)P.p.M * P.nH / 1.2e10 + 30.0 * (n2 * 1e-11 + 3e-5);
    }
    b->order.resize(n_plans);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    *out = b;
    return FIRM_OK;
}

int firm_batch_run(firm_batch_t b, const firm_batch_item* items, int iters, int flags) {
    if (!b || iters < 0 || iters >= kMaxHist || (flags & ~(FIRM_BATCH_GRAPH | FIRM_BATCH_PERSISTENT))) return FIRM_EINVAL;
    const int st = check_items(*b, items);
    if (st != FIRM_OK) return st;
    b->last_tol = 0.0;
    return run(*b, items, iters, flags);
}

int firm_batch_set_network(firm_batch_t b, const void* params_bf16, const float* params) {
    if (!b || (params_bf16 == nullptr) != (params == nullptr)) return FIRM_EINVAL;
    if (params && (!dev_ptr(params_bf16) || !dev_ptr(params))) return FIRM_EINVAL;
    b->net_bf16 = params_bf16;
    b->net = params;
    return FIRM_OK;
}

int firm_batch_solve(firm_batch_t b, const firm_batch_item* items, int max_iter, double rel_tol, int flags) {
    if (!b || max_iter < 0 || max_iter >= kMaxHist || !(rel_tol >= 0.0) ||
        (flags & ~(FIRM_BATCH_GRAPH | FIRM_BATCH_PERSISTENT | FIRM_BATCH_LEARNED)))
        return FIRM_EINVAL;
    if ((flags & FIRM_BATCH_LEARNED) && !b->net) return FIRM_ESTATE;
    if (!(flags & FIRM_BATCH_LEARNED))
        for (auto* h : b->plans)
            if (h->P.pc_mode == FIRM_PRECOND_BINNED) return FIRM_EINVAL;     // needs the host per plan
    int st = check_items(*b, items);
    if (st != FIRM_OK) return st;
    st = run(*b, items, max_iter, flags | kSolveFront, rel_tol);
    if (st != FIRM_OK) return st;
    st = run_cg_chunks(*b, max_iter, (flags & FIRM_BATCH_GRAPH) != 0);
    if (st != FIRM_OK) return st;
    for (int i = 0; i < b->n; ++i) {
        const Plan& P = b->plans[i]->P;
        if (cudaMemcpyAsync(items[i].x, P.ws.x, sizeof(float) * P.N * P.N * P.N, cudaMemcpyDeviceToDevice,
                            b->main) != cudaSuccess)
            return FIRM_ECUDA;
    }
    if (cudaEventRecord(b->ev_out, b->main) != cudaSuccess || cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess)
        return FIRM_ECUDA;
    b->last_tol = rel_tol;
    return FIRM_OK;
}

int firm_batch_wait(firm_batch_t b, int* status, int* iters) {
    if (!b) return FIRM_EINVAL;
    if (!b->ran) return FIRM_ESTATE;
    if (cudaStreamSynchronize(b->main) != cudaSuccess) return FIRM_ECUDA;
    int first = FIRM_OK;
    for (int i = 0; i < b->n; ++i) {
        Plan& P = b->plans[i]->P;
        CgState s;
        int flag = 0;
        if (cudaMemcpy(&s, P.ws.cg, sizeof(CgState), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&flag, P.ws.counters + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return FIRM_ECUDA;
        if (flag && cudaMemset(P.ws.counters + 2, 0, sizeof(int)) != cudaSuccess) return FIRM_ECUDA;
        int sti = flag ? FIRM_EINTERNAL : s.status;
        if (sti == FIRM_OK && b->last_tol > 0.0 && !(s.rr >= 0.0 && std::sqrt(s.rr) <= s.tol)) sti = FIRM_ENOTCONV;
        P.have_kernel = P.have_rhs = true;
        P.pc_ready = false;
        P.cg_iters = s.it;
        if (status) status[i] = sti;
        if (iters) iters[i] = s.it;
        if (sti != FIRM_OK && first == FIRM_OK) first = sti;
    }
    return first;
}

int firm_batch_set_config(firm_batch_t b, int n_streams, int chunk) {
    if (!b || n_streams < 1 || n_streams > (int)b->streams.size() || chunk < kMinChunk || chunk > kChunk ||
        chunk % 256 != 0)
        return FIRM_EINVAL;
    b->n_streams = std::min(n_streams, b->n);
    b->chunk = chunk;
    return FIRM_OK;
}

int firm_batch_get_config(firm_batch_t b, int* n_streams, int* chunk) {
    if (!b) return FIRM_EINVAL;
    if (n_streams) *n_streams = b->n_streams;
    if (chunk) *chunk = b->chunk;
    return FIRM_OK;
}

int firm_batch_tune(firm_batch_t b, const firm_batch_item* items, int iters, int flags, double* ms_out) {
    if (!b || iters < 0 || iters >= kMaxHist || (flags & ~(FIRM_BATCH_GRAPH | FIRM_BATCH_PERSISTENT))) return FIRM_EINVAL;
    int st = check_items(*b, items);
    if (st != FIRM_OK) return st;
    auto time_one = [&](int ns, int ch, double* ms) -> int {
        b->n_streams = std::min(ns, b->n);
        b->chunk = ch;
        int r = run(*b, items, iters, flags);
        if (r != FIRM_OK) return r;
        if (cudaEventRecord(b->ev_t0, b->main) != cudaSuccess) return FIRM_ECUDA;
        r = run(*b, items, iters, flags);
        if (r != FIRM_OK) return r;
        if (cudaEventRecord(b->ev_t1, b->main) != cudaSuccess || cudaEventSynchronize(b->ev_t1) != cudaSuccess)
            return FIRM_ECUDA;
        float f = 0.f;
        if (cudaEventElapsedTime(&f, b->ev_t0, b->ev_t1) != cudaSuccess) return FIRM_ECUDA;
        *ms = f;
        return FIRM_OK;
    };
    const int max_s = (int)b->streams.size();
    int best_s = std::min(8, max_s), best_c = kChunk;
    double best = 1e300, ms = 0.0;
    // work-item size first (at a middling stream count), then the stream count
    for (int ch : {2048, 4096, 8192}) {
        st = time_one(best_s, ch, &ms);
        if (st != FIRM_OK) return st;
        if (ms < best) { best = ms; best_c = ch; }
    }
    for (int ns : {1, 2, 4, 8, 16, 32, 64}) {
        if (ns > max_s || ns > b->n || ns == std::min(8, max_s)) continue;
        st = time_one(ns, best_c, &ms);
        if (st != FIRM_OK) return st;
        if (ms < best) { best = ms; best_s = ns; }
    }
    b->n_streams = std::min(best_s, b->n);
    b->chunk = best_c;
    if (ms_out) *ms_out = best;
    return FIRM_OK;
}

int firm_batch_launch_count(firm_batch_t b, long long* out) {
    if (!b || !out) return FIRM_EINVAL;
    *out = b->launches_per_run;
    return FIRM_OK;
}

void firm_batch_destroy(firm_batch_t b) {
    if (!b) return;
    if (b->main) cudaStreamSynchronize(b->main);
    drop_graph(*b);
    drop_cg_graph(*b);
    for (auto s : b->streams)
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    for (auto e : b->ev_join)
        if (e) cudaEventDestroy(e);
    for (auto e : b->ev_fork)
        if (e) cudaEventDestroy(e);
    if (b->ev_t0) cudaEventDestroy(b->ev_t0);
    if (b->ev_t1) cudaEventDestroy(b->ev_t1);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->main) cudaStreamDestroy(b->main);
    delete b;
}

}  // extern "C"
