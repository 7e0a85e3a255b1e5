// Batched reconstructions: many independent problems of different shapes in
// one launch.  Each request's whole reconstruction (its own plan, so its own
// factors, tiles and workspace) is captured into a child graph; the children
// are independent nodes of one parent graph, so the GPU runs them
// concurrently and one cudaGraphLaunch replays the whole batch.  The parent
// graph is cached while the requests (plans, pointers, parameters) repeat and
// each plan is the same plan (serial) in the same configuration (generation).
// A request's result does not depend on the others: every request is
// computed by exactly the kernels, tiles and summation order it would use
// alone.
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

struct mri_batch {
    std::vector<mri_request> key;
    std::vector<std::pair<uint64_t, uint64_t>> plan_ids;  // (serial, config_gen) of each request's plan
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;
    long long launches = 0;  // kernels in one replay
};

namespace mri {
namespace {

bool same_request(const mri_request &a, const mri_request &b) {
    return a.plan == b.plan && a.kspace == b.kspace && a.coil_maps == b.coil_maps && a.image_out == b.image_out &&
           a.params.lambda == b.params.lambda && a.params.beta == b.params.beta &&
           a.params.admm_iters == b.params.admm_iters && a.params.cg_iters == b.params.cg_iters &&
           a.params.rtol == b.params.rtol && a.params.atol == b.params.atol;
}

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

void drop(mri_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key.clear();
    b->plan_ids.clear();
    b->launches = 0;
}

}  // namespace
}  // namespace mri

using namespace mri;

extern "C" {

MRI_API int mri_batch_create(mri_batch **out) {
    if (!out) return fail(MRI_ERR_INVALID, "batch output pointer is null");
    mri_batch *b = new mri_batch();
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return fail(MRI_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    *out = b;
    return MRI_OK;
}

MRI_API int mri_batch_destroy(mri_batch *b) {
    if (!b) return MRI_OK;
    cudaDeviceSynchronize();
    drop(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
    return MRI_OK;
}

MRI_API long long mri_batch_launch_count(const mri_batch *b) { return b ? b->launches : 0; }

MRI_API int mri_batch_reconstruct(mri_batch *b, int n, const mri_request *reqs, mri_stream_t stream) {
    NvtxRange range("mri_batch_reconstruct");
    if (!b || n <= 0 || !reqs) return fail(MRI_ERR_INVALID, "null batch, empty request list or null requests");
    for (int q = 0; q < n; ++q) {
        const mri_request &r = reqs[q];
        const int rc = check_admm_args(r.plan, r.kspace, r.coil_maps, &r.params, r.image_out);
        if (rc != MRI_OK) return fail(rc, "request " + std::to_string(q) + ": " + mri_last_error());
        if (r.plan->timing) return fail(MRI_ERR_INVALID, "request " + std::to_string(q) + ": plan has timing on");
        for (int t = 0; t < q; ++t)
            if (reqs[t].plan == r.plan)
                return fail(MRI_ERR_INVALID, "requests " + std::to_string(t) + " and " + std::to_string(q) +
                                                 " share a plan (each needs its own workspace)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    bool hit = b->exec && (int)b->key.size() == n;
    for (int q = 0; hit && q < n; ++q)
        hit = same_request(b->key[q], reqs[q]) &&
              b->plan_ids[q] == std::make_pair(reqs[q].plan->serial, reqs[q].plan->config_gen);
    if (!hit) {
        drop(b);
        cudaGraph_t parent = nullptr;
        cudaError_t e = cudaGraphCreate(&parent, 0);
        if (e != cudaSuccess) return fail(MRI_ERR_CUDA, std::string("cudaGraphCreate: ") + cudaGetErrorString(e));
        long long launches = 0;
        for (int q = 0; q < n && e == cudaSuccess; ++q) {
            const mri_request &r = reqs[q];
            const long long l0 = r.plan->launches;
            e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            // the items run concurrently: CG steps as ordinary kernels (a
            // cooperative grid would wait for the whole GPU), same results
            const int rc = enqueue_admm(r.plan, r.kspace, r.coil_maps, &r.params, r.image_out, nullptr, nullptr,
                                        b->capture, AdmmWarm(), false);
            cudaGraph_t child = nullptr;
            e = cudaStreamEndCapture(b->capture, &child);
            if (rc != MRI_OK || e != cudaSuccess) {
                if (child) cudaGraphDestroy(child);
                cudaGraphDestroy(parent);
                return rc != MRI_OK ? rc : fail(MRI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            }
            launches += r.plan->launches - l0;
            cudaGraphNode_t node;
            e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, child);
            cudaGraphDestroy(child);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, parent, 0);
        cudaGraphDestroy(parent);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return fail(MRI_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        }
        b->key.assign(reqs, reqs + n);
        b->plan_ids.clear();
        for (int q = 0; q < n; ++q) b->plan_ids.emplace_back(reqs[q].plan->serial, reqs[q].plan->config_gen);
        b->launches = launches;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return fail(MRI_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    return MRI_OK;
}

}  // extern "C"
