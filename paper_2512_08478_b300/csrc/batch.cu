// vis_render_batch -- many assets seen by many cameras in one call (the paper renders
// several models per frame with one global sort, Algorithm 1; here each image is an
// independent render, and the batch is one CUDA graph).
//
// Plan: images are assigned to `lanes` (streams forked from the batch's origin stream)
// by longest-processing-time scheduling on the estimated cost (Gaussians + pixels);
// each lane renders its images one after another in its own workspace slice, and
// after every image a one-thread kernel copies the slice's status (key count, error
// bits) into the image's status word, so no image's error is lost. The whole fork /
// render / join sequence is captured once into a CUDA graph and replayed by later
// calls with the same arguments: lanes become concurrent graph branches, so small
// images of small assets overlap instead of leaving the GPU idle between launches.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vis_internal.cuh"

struct vis_batch {
    int lanes = 0;
    cudaStream_t origin = nullptr;   // the graph is captured on and launched from this stream
    cudaEvent_t in_ev = nullptr, out_ev = nullptr;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;   // serialised arguments of the captured graph
    int device = -1;
};

namespace vis {

__global__ void copy_status_kernel(const Ctrl* __restrict__ ctrl, uint32_t* __restrict__ status) {
    status[0] = ctrl->num_keys;
    status[1] = ctrl->error;
}

}  // namespace vis

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// status words live at the start of the batch workspace: 2 x uint32 per image
size_t status_bytes(int n_images) { return align256(sizeof(uint32_t) * 2 * (size_t)n_images); }

struct Plan {
    std::vector<int> lane_of;            // image -> lane
    std::vector<std::vector<int>> order; // lane -> images in render order
    size_t slice_bytes = 0;
};

vis_status fail_b(vis_status s, const std::string& m) {
    vis::set_last_error(m.c_str());
    return s;
}

Plan make_plan(const vis_scene_t* scenes, const int* cam_scene, const int* W, const int* H, int n_images, int lanes,
               size_t slice_bytes) {
    Plan p;
    p.lane_of.assign(n_images, 0);
    p.order.assign(lanes, {});
    std::vector<double> cost(n_images), load(lanes, 0.0);
    std::vector<int> idx(n_images);
    for (int i = 0; i < n_images; ++i) {
        idx[i] = i;
        cost[i] = (double)vis::scene_size(scenes[cam_scene[i]]) + 4.0 * (double)W[i] * H[i];
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i : idx) {
        int best = 0;
        for (int l = 1; l < lanes; ++l)
            if (load[l] < load[best]) best = l;
        p.lane_of[i] = best;
        p.order[best].push_back(i);
        load[best] += cost[i];
    }
    p.slice_bytes = slice_bytes;
    return p;
}

void append(std::vector<unsigned char>& k, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    k.insert(k.end(), c, c + n);
}

}  // namespace

extern "C" {

vis_status vis_batch_create(int lanes, vis_batch_t* out) {
    if (!out) return fail_b(VIS_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (lanes < 1 || lanes > 64) return fail_b(VIS_ERR_INVALID_ARG, "lanes must be in [1, 64]");
    vis_batch* b = new (std::nothrow) vis_batch;
    if (!b) return fail_b(VIS_ERR_INVALID_ARG, "out of host memory");
    b->lanes = lanes;
    cudaGetDevice(&b->device);
    b->streams.resize(lanes);
    b->join_ev.resize(lanes);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->in_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->out_ev, cudaEventDisableTiming);
    for (int l = 0; l < lanes && e == cudaSuccess; ++l) {
        e = cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[l], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        vis_batch_destroy(b);
        return fail_b(VIS_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    *out = b;
    vis::set_last_error("");
    return VIS_OK;
}

void vis_batch_destroy(vis_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto ev : b->join_ev) if (ev) cudaEventDestroy(ev);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->in_ev) cudaEventDestroy(b->in_ev);
    if (b->out_ev) cudaEventDestroy(b->out_ev);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

vis_status vis_batch_workspace_size(const vis_scene_t* scenes, int n_scenes, const int* cam_scene, const int* W,
                                    const int* H, int n_images, int lanes, int64_t key_capacity,
                                    const vis_render_opts* opts, size_t* bytes) {
    if (!scenes || !cam_scene || !W || !H || !bytes) return fail_b(VIS_ERR_INVALID_ARG, "null argument");
    if (n_images < 1 || n_scenes < 1 || lanes < 1) return fail_b(VIS_ERR_INVALID_ARG, "empty batch");
    size_t slice = 0;
    for (int i = 0; i < n_images; ++i) {
        if (cam_scene[i] < 0 || cam_scene[i] >= n_scenes || !scenes[cam_scene[i]])
            return fail_b(VIS_ERR_INVALID_ARG, "cam_scene out of range");
        size_t b = 0;
        vis_status st = vis_workspace_size(vis::scene_size(scenes[cam_scene[i]]), W[i], H[i], key_capacity, opts, &b);
        if (st) return st;
        if (b > slice) slice = b;
    }
    *bytes = status_bytes(n_images) + (size_t)lanes * align256(slice);
    vis::set_last_error("");
    return VIS_OK;
}

vis_status vis_render_batch(vis_batch_t b, const vis_scene_t* scenes, int n_scenes, const vis_camera* cams,
                            const int* cam_scene, const int* W, const int* H, int n_images, const float bg[3],
                            float* const* out_rgb, float* const* out_alpha, void* ws, size_t ws_bytes,
                            const vis_render_opts* opts, void* stream_) {
    if (!b) return fail_b(VIS_ERR_INVALID_ARG, "batch handle is null");
    if (!scenes || !cams || !cam_scene || !W || !H || !bg || !out_rgb || !out_alpha || !ws)
        return fail_b(VIS_ERR_INVALID_ARG, "null argument");
    if (n_images < 1 || n_scenes < 1) return fail_b(VIS_ERR_INVALID_ARG, "empty batch");
    const size_t sb = status_bytes(n_images);
    if (ws_bytes <= sb) return fail_b(VIS_ERR_INVALID_ARG, "batch workspace too small");
    const size_t slice = ((ws_bytes - sb) / b->lanes) / 256 * 256;
    for (int i = 0; i < n_images; ++i)
        if (cam_scene[i] < 0 || cam_scene[i] >= n_scenes || !scenes[cam_scene[i]])
            return fail_b(VIS_ERR_INVALID_ARG, "cam_scene out of range");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    char* w = static_cast<char*>(ws);

    // arguments that the captured graph depends on
    std::vector<unsigned char> key;
    vis_render_opts o;
    vis_default_opts(&o);
    if (opts) o = *opts;
    append(key, &o, sizeof(o));
    append(key, &ws, sizeof(ws));
    append(key, &ws_bytes, sizeof(ws_bytes));
    append(key, bg, 3 * sizeof(float));
    append(key, &n_images, sizeof(n_images));
    for (int i = 0; i < n_images; ++i) {
        append(key, &cams[i], sizeof(vis_camera));
        append(key, &W[i], sizeof(int));
        append(key, &H[i], sizeof(int));
        append(key, &out_rgb[i], sizeof(float*));
        append(key, &out_alpha[i], sizeof(float*));
        vis::append_scene_key(key, scenes[cam_scene[i]]);
    }
    if (!b->exec || key != b->key) {
        // validate every image before capturing (errors cannot be returned from inside)
        for (int i = 0; i < n_images; ++i) {
            vis_ws_layout L;
            vis_status st = vis_workspace_layout(vis::scene_size(scenes[cam_scene[i]]), W[i], H[i], slice, &o, &L);
            if (st) return st;
        }
        const Plan plan = make_plan(scenes, cam_scene, W, H, n_images, b->lanes, slice);
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        vis_status st = VIS_OK;
        cudaEventRecord(b->fork_ev, b->origin);
        for (int l = 0; l < b->lanes; ++l) cudaStreamWaitEvent(b->streams[l], b->fork_ev, 0);
        for (int l = 0; l < b->lanes && st == VIS_OK; ++l) {
            char* sw = w + sb + (size_t)l * slice;
            for (int i : plan.order[l]) {
                st = vis_render(scenes[cam_scene[i]], &cams[i], W[i], H[i], bg, out_rgb[i], out_alpha[i], sw, slice,
                                &o, b->streams[l]);
                if (st) break;
                vis::copy_status_kernel<<<1, 1, 0, b->streams[l]>>>(reinterpret_cast<const vis::Ctrl*>(sw),
                                                                   reinterpret_cast<uint32_t*>(w) + 2 * i);
            }
        }
        for (int l = 0; l < b->lanes; ++l) {
            cudaEventRecord(b->join_ev[l], b->streams[l]);
            cudaStreamWaitEvent(b->origin, b->join_ev[l], 0);
        }
        e = cudaStreamEndCapture(b->origin, &graph);
        if (st) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { b->exec = nullptr; return fail_b(VIS_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
        b->key = key;
    }
    // order the graph after the caller's prior work and the caller's later work after it
    cudaError_t e = cudaEventRecord(b->in_ev, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->in_ev, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(b->out_ev, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->out_ev, 0);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    vis::set_last_error("");
    return VIS_OK;
}

vis_status vis_batch_check(const void* ws, int n_images, void* stream_, int64_t* max_keys) {
    if (!ws || n_images < 1) return fail_b(VIS_ERR_INVALID_ARG, "null workspace or empty batch");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, cudaGetErrorString(e));
    std::vector<uint32_t> st(2 * (size_t)n_images);
    e = cudaMemcpy(st.data(), ws, st.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, cudaGetErrorString(e));
    uint32_t mk = 0, err = 0;
    for (int i = 0; i < n_images; ++i) {
        if (st[2 * i] > mk) mk = st[2 * i];
        err |= st[2 * i + 1];
    }
    if (max_keys) *max_keys = mk;
    if (err & vis::kErrCapacity)
        return fail_b(VIS_ERR_CAPACITY, "an image of the batch produced more keys than its workspace slice holds");
    if (err & vis::kErrTimeout) return fail_b(VIS_ERR_TIMEOUT, "a device spin wait timed out");
    vis::set_last_error("");
    return VIS_OK;
}

}  // extern "C"
