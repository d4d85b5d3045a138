// Autotuner for the planner's free parameters (Sec. 3.17: after the memory
// capacity has fixed what it must, the few remaining choices are made by
// measurement): the base-case path and the Strassen depth per shape.
//
// Small products are timed whole on synthetic operands. For large ones the
// leaf products of each candidate are timed on a leaf-shaped proxy (at most
// 16384 bits a side, as many leaves as fit in 1 GiB, in one batched launch)
// and scaled to the leaf count and size; the streaming passes (transpose,
// XOR passes) are charged the plan's bytes at the measured device copy
// bandwidth. The kernels' running time does not depend on the bits, so any
// operand contents serve.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace bmm {

namespace {

struct Key {
    int dev, op;
    int64_t m, k, n;
    bool operator<(const Key& o) const {
        return std::tie(dev, op, m, k, n) < std::tie(o.dev, o.op, o.m, o.k, o.n);
    }
};

std::mutex g_tune_mu;
std::map<Key, std::pair<int, int>> g_choice;  // (path, depth)

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Arbitrary bits for timing: a multiplicative hash of the word index.
__global__ void timing_fill_kernel(uint64_t* p, int64_t words, uint64_t salt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = ((uint64_t)i + salt) * 6364136223846793005ull + 1442695040888963407ull;
        p[i] = z ^ (z >> 29);
    }
}

// Stream-ordered scratch freed on scope exit.
struct Buf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    bmm_status get(uint64_t bytes, cudaStream_t st) {
        s = st;
        if (bytes == 0) return BMM_OK;
        const cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return cuda_fail(e);
        }
        return BMM_OK;
    }
    uint64_t* w() const { return (uint64_t*)p; }
    ~Buf() {
        if (p) cudaFreeAsync(p, s);
    }
};

bmm_status fill(uint64_t* p, uint64_t words, uint64_t salt, cudaStream_t s) {
    if (words == 0) return BMM_OK;
    const uint64_t want = (words + 255) / 256;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)sm_count() * 8);
    timing_fill_kernel<<<blocks, 256, 0, s>>>(p, (int64_t)words, salt);
    BMM_CUDA_TRY(cudaGetLastError());
    return BMM_OK;
}

// Mean milliseconds of `reps` runs of f, after one untimed run.
template <class F>
bmm_status time_runs(F&& f, int reps, cudaStream_t s, double* ms) {
    bmm_status st = f();
    if (st != BMM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BMM_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce);
    }
    ce = cudaEventRecord(e0, s);
    for (int r = 0; st == BMM_OK && ce == cudaSuccess && r < reps; r++) st = f();
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float t = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != BMM_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(ce);
    *ms = (double)t / reps;
    return BMM_OK;
}

// Device-to-device copy bandwidth (bytes read + written per second).
bmm_status copy_bandwidth(cudaStream_t s, double* bytes_per_s) {
    size_t fr = 0, tot = 0;
    BMM_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    uint64_t bytes = 256ull << 20;
    while (bytes > (4ull << 20) && 2 * bytes > fr / 4) bytes /= 2;
    Buf a, b;
    bmm_status st = a.get(bytes, s);
    if (st == BMM_OK) st = b.get(bytes, s);
    if (st != BMM_OK) return st;
    double ms = 0;
    st = time_runs(
        [&]() -> bmm_status {
            BMM_CUDA_TRY(cudaMemcpyAsync(b.p, a.p, bytes, cudaMemcpyDeviceToDevice, s));
            return BMM_OK;
        },
        3, s, &ms);
    if (st != BMM_OK) return st;
    *bytes_per_s = 2.0 * (double)bytes / (ms * 1e-3);
    return BMM_OK;
}

struct Cand {
    int path, depth;
    Plan plan;
    double ms;
};

int64_t pow7(int d) {
    int64_t r = 1;
    while (d-- > 0) r *= 7;
    return r;
}

// Leaf products of one candidate, timed on a proxy and scaled.
bmm_status model_leaves(int op, const Cand& c, cudaStream_t s, double* ms) {
    const int d = c.depth;
    const int64_t ml = c.plan.m >> d, kl = c.plan.kp >> d, nl = c.plan.n >> d;
    const int64_t mp = std::min<int64_t>(ml, 16384), kp = std::min<int64_t>(kl, 16384),
                  np = std::min<int64_t>(nl, 16384);
    const uint64_t a = (uint64_t)mp * kp / 8, b = (uint64_t)np * kp / 8, cc = (uint64_t)mp * np / 8;
    const int64_t leaves = pow7(d);
    const int64_t cnt =
        std::max<int64_t>(1, std::min<int64_t>(leaves, (int64_t)((1ull << 30) / (a + b + cc))));
    Buf A, B, C;
    bmm_status st = A.get(cnt * a, s);
    if (st == BMM_OK) st = B.get(cnt * b, s);
    if (st == BMM_OK) st = C.get(cnt * cc, s);
    if (st == BMM_OK) st = fill(A.w(), cnt * a / 8, 1, s);
    if (st == BMM_OK) st = fill(B.w(), cnt * b / 8, 2, s);
    if (st != BMM_OK) return st;
    double t = 0;
    st = time_runs(
        [&]() {
            return run_base_product_batched(op, c.path, A.w(), kp / 64, (int64_t)(a / 8), B.w(),
                                            kp / 64, (int64_t)(b / 8), C.w(), np / 64,
                                            (int64_t)(cc / 8), cnt, mp, kp, np, s);
        },
        2, s, &t);
    if (st != BMM_OK) return st;
    *ms = t * ((double)leaves / (double)cnt) *
          ((double)ml * (double)kl * (double)nl / ((double)mp * (double)kp * (double)np));
    return BMM_OK;
}

}  // namespace

bool tuned_choice(int op, int64_t m, int64_t k, int64_t n, int* path, int* depth) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_choice.find(Key{current_device(), op, m, k, n});
    if (it == g_choice.end()) return false;
    *path = it->second.first;
    *depth = it->second.second;
    return true;
}

}  // namespace bmm

using namespace bmm;

extern "C" bmm_status bmm_autotune(int32_t op, int64_t m, int64_t k, int64_t n, uint32_t flags,
                                   bmm_stream_t stream, bmm_tune_result* result) {
    if (!result || (op != OP_GF2 && op != OP_BOOL)) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    if (flags & ~BMM_TUNE_MODEL) return BMM_ERR_INVALID;
    const cudaStream_t s = (cudaStream_t)stream;

    // candidates the planner accepts, with their plans (serial depth by the
    // planner's memory rule)
    std::vector<int> paths;
    if (tc_fp4_available()) paths.push_back(BMM_PATH_TC_FP4_PAIR);
    if (tc_pair_available()) paths.push_back(BMM_PATH_TC_FP8_PAIR);
    if (tc_path_available()) paths.push_back(BMM_PATH_TC_FP8);
    paths.push_back(BMM_PATH_POPC);
    std::vector<Cand> cands;
    for (int path : paths) {
        for (int d = 0; d <= (op == OP_GF2 ? 4 : 0); d++) {
            if (d > 0 && ((m >> d) < 256 || (k >> d) < 256 || (n >> d) < 256)) continue;
            bmm_opts o;
            bmm_opts_default(&o);
            o.path = path;
            o.strassen_depth = d;
            Cand c{path, d, Plan{}, 0.0};
            if (make_plan(op, m, k, n, &o, &c.plan) != BMM_OK) continue;
            cands.push_back(c);
        }
    }
    if (cands.empty()) return BMM_ERR_UNSUPPORTED;

    size_t fr = 0, tot = 0;
    BMM_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    const uint64_t ab = (uint64_t)m * k / 8, bb = (uint64_t)k * n / 8, cb = (uint64_t)m * n / 8;
    uint64_t maxws = 0;
    for (const Cand& c : cands) maxws = std::max(maxws, c.plan.workspace_bytes);
    const double cubic_s = 2.0 * (double)m * (double)k * (double)n / 3.0e15;
    const bool whole =
        !(flags & BMM_TUNE_MODEL) && ab + bb + cb + maxws <= fr / 4 && cubic_s < 0.1;

    bmm_status st = BMM_OK;
    if (whole) {
        Buf A, B, C, W;
        st = A.get(ab, s);
        if (st == BMM_OK) st = B.get(bb, s);
        if (st == BMM_OK) st = C.get(cb, s);
        if (st == BMM_OK) st = W.get(maxws, s);
        if (st == BMM_OK) st = fill(A.w(), ab / 8, 3, s);
        if (st == BMM_OK) st = fill(B.w(), bb / 8, 4, s);
        for (size_t i = 0; st == BMM_OK && i < cands.size(); i++) {
            Cand& c = cands[i];
            st = time_runs([&]() { return execute_plan(c.plan, A.w(), B.w(), C.w(), W.p, s); }, 2,
                           s, &c.ms);
        }
    } else {
        double bw = 0;
        st = copy_bandwidth(s, &bw);
        for (size_t i = 0; st == BMM_OK && i < cands.size(); i++) {
            Cand& c = cands[i];
            double leaves_ms = 0;
            st = model_leaves(op, c, s, &leaves_ms);
            c.ms = leaves_ms + (double)plan_pass_bytes(c.plan) / bw * 1e3;
        }
    }
    if (st == BMM_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (st != BMM_OK) return st;

    const Cand* best = &cands[0];
    for (const Cand& c : cands)
        if (c.ms < best->ms) best = &c;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_choice[Key{current_device(), op, m, k, n}] = {best->path, best->depth};
    }
    bmm_opts_default(&result->best);
    result->best.path = best->path;
    result->best.strassen_depth = best->depth;
    result->est_ms = best->ms;
    result->measured = whole ? 1 : 0;
    result->candidates = (int32_t)cands.size();
    return BMM_OK;
}

extern "C" void bmm_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_choice.clear();
}
