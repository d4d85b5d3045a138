// Host layer: products whose operands and result live in host memory
// (Secs. 3.12-3.14 and Alg. 3, for one accelerator fed over its host link).
//
// Binary product with host levels (host_depth d >= 1): the host generates
// the 7^d sub-instances T_h = xi_h(A), S_h = eta_h(B) by aggregating the
// quadrant blocks their combined standard-basis masks select over all d
// levels at once (Eq. igen, with the basis change folded in: xi = alpha phi,
// eta = beta psi), the GPU solves each (its own plan: tensor-core base case,
// Strassen below), and the host aggregates every solution into the C blocks
// zeta = chi gamma selects (Eq. iagg). One pipeline with four roles, as in
// Alg. 3 for N = 1: a generator thread fills pinned T/S staging buffers,
// the calling thread uploads, launches and downloads on three streams, and
// an aggregator thread folds the downloaded Q_h into C; every buffer is
// double-buffered, so generation, transfer, compute and aggregation of
// neighbouring sub-instances overlap.
//
// Otherwise (Boolean products, which have no additive inverse, or host_depth
// 0), C is cut into blocks that fit the device: each block product streams
// its row panel of A (uploaded once per block row) and its column panel of B
// straight from the caller's arrays and writes its C block straight back.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "plan.h"
#include "slp.h"

namespace bmm {

namespace {

constexpr uint64_t SLACK = 8ull << 20;  // allocator rounding and the planner's small buffers

uint64_t pow7u(int d) {
    uint64_t r = 1;
    while (d-- > 0) r *= 7;
    return r;
}

bool host_divisible(int64_t m, int64_t k, int64_t n, int d) {
    const int64_t unit = (int64_t)64 << d;
    return m % unit == 0 && k % unit == 0 && n % unit == 0;
}

// Device scratch of one product's plan, by the planner's rules (depth from
// the options or the automatic rule, the innermost level inside the
// CUDA-core kernel when asked for, depth-first levels above two merged ones,
// k padded for the tensor paths), without asking the device.
uint64_t product_scratch(int op, int64_t m, int64_t k, int64_t n, const bmm_opts& o) {
    int d = 0;
    if (op == OP_GF2) {
        if (o.strassen_depth >= 0) {
            d = o.strassen_depth;
        } else {
            while (d < 4 && m % ((int64_t)64 << (d + 1)) == 0 && k % ((int64_t)64 << (d + 1)) == 0 &&
                   n % ((int64_t)64 << (d + 1)) == 0 && (m >> (d + 1)) >= 8192 &&
                   (k >> (d + 1)) >= 8192 && (n >> (d + 1)) >= 8192)
                d++;
        }
    }
    // the path the device plan resolves AUTO to (the CUDA cores where the
    // device has no tensor-core path, and without a device)
    const int path = o.path == BMM_PATH_AUTO ? auto_path() : o.path;
    const bool kl = o.kernel_level == 1 && d > 0 &&
                    (path == BMM_PATH_POPC || path == BMM_PATH_TC_FP4_PAIR);
    const int od = kl ? d - 1 : d;
    const int serial = od > 2 ? od - 2 : 0;
    const int64_t unit = (int64_t)(kl ? 512 : 128) << d;
    const int64_t kp = path == BMM_PATH_POPC ? k : (k + unit - 1) / unit * unit;
    return workspace_padded(m, k, kp, n, od, serial);
}

struct HostPlan {
    int op = OP_GF2;
    int host_depth = 0;
    int64_t m = 0, k = 0, n = 0;
    int64_t bm = 0, bn = 0;  // device product: bm x k' x bn (k' = k >> host_depth)
    int64_t count = 0;
    uint64_t device_bytes = 0, staging_bytes = 0, upload_bytes = 0, download_bytes = 0;
};

uint64_t strassen_device_bytes(int op, int64_t sm, int64_t sk, int64_t sn, const bmm_opts& o) {
    const uint64_t t = (uint64_t)sm * sk / 8, s = (uint64_t)sk * sn / 8, q = (uint64_t)sm * sn / 8;
    return 2 * (t + s + q) + product_scratch(op, sm, sk, sn, o) + SLACK;
}

uint64_t blocked_device_bytes(int op, int64_t bm, int64_t k, int64_t bn, const bmm_opts& o) {
    const uint64_t a = (uint64_t)bm * k / 8, b = (uint64_t)k * bn / 8, c = (uint64_t)bm * bn / 8;
    return 2 * (a + b + c) + product_scratch(op, bm, k, bn, o) + SLACK;
}

bmm_status host_plan(int op, int64_t m, int64_t k, int64_t n, const bmm_host_opts& ho,
                     uint64_t budget, HostPlan* out) {
    HostPlan p;
    p.op = op;
    p.m = m;
    p.k = k;
    p.n = n;
    const bmm_opts& o = ho.device;
    const uint64_t ab = (uint64_t)m * k / 8, bb = (uint64_t)k * n / 8, cb = (uint64_t)m * n / 8;
    if (ho.host_depth > 0 && op != OP_GF2) return BMM_ERR_INVALID;  // no additive inverse
    if (ho.host_depth > 4) return BMM_ERR_UNSUPPORTED;
    int d = ho.host_depth;
    if (d < 0) {
        // the fewest host levels whose sub-instances fit the device; none when
        // the whole product fits, blocks of C when no level count does
        d = 0;
        if (op == OP_GF2 && blocked_device_bytes(op, m, k, n, o) > budget) {
            for (int t = 1; t <= 4 && host_divisible(m, k, n, t); t++)
                if (strassen_device_bytes(op, m >> t, k >> t, n >> t, o) <= budget) {
                    d = t;
                    break;
                }
        }
    }
    if (d > 0) {
        if (!host_divisible(m, k, n, d)) return BMM_ERR_UNSUPPORTED;
        const int64_t sm = m >> d, sk = k >> d, sn = n >> d;
        p.host_depth = d;
        p.bm = sm;
        p.bn = sn;
        p.count = (int64_t)pow7u(d);
        p.device_bytes = strassen_device_bytes(op, sm, sk, sn, o);
        if (p.device_bytes > budget) return BMM_ERR_NOMEM;
        const uint64_t t = (uint64_t)sm * sk / 8, s = (uint64_t)sk * sn / 8, q = (uint64_t)sm * sn / 8;
        p.staging_bytes = 2 * (t + s + q);
        p.upload_bytes = (uint64_t)p.count * (t + s);
        p.download_bytes = (uint64_t)p.count * q;
        *out = p;
        return BMM_OK;
    }
    // blocks of C, each with full k: halve the longer side until one fits
    int64_t bm = m, bn = n;
    while (blocked_device_bytes(op, bm, k, bn, o) > budget) {
        if (bm >= bn && bm > 256)
            bm = (bm / 2 + 63) / 64 * 64;
        else if (bn > 256)
            bn = (bn / 2 + 63) / 64 * 64;
        else
            return BMM_ERR_NOMEM;
    }
    const int64_t rm = (m + bm - 1) / bm, rn = (n + bn - 1) / bn;
    p.host_depth = 0;
    p.bm = bm;
    p.bn = bn;
    p.count = rm * rn;
    p.device_bytes = blocked_device_bytes(op, bm, k, bn, o);
    p.upload_bytes = ab + (uint64_t)rm * bb;
    p.download_bytes = cb;
    *out = p;
    return BMM_OK;
}

// ---------------------------------------------------------------- host passes
int host_threads(const bmm_host_opts& ho) {
    if (ho.threads > 0) return ho.threads;
    const unsigned h = std::thread::hardware_concurrency();
    return h > 0 ? (int)h : 1;
}

// Persistent workers for one host role's passes (a pass runs part i of n on
// worker i, the calling thread being worker 0, and returns when all parts
// are done): threads are started once per product, not once per pass.
class Pool {
  public:
    explicit Pool(int n) : size_(std::max(1, n)) {
        for (int i = 1; i < size_; i++) th_.emplace_back([this, i]() { worker(i); });
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    int size() const { return size_; }
    // f(i) for i in [0, parts), parts <= size()
    void run(int parts, const std::function<void(int)>& f) {
        if (parts <= 1 || th_.empty()) {
            for (int i = 0; i < parts; i++) f(i);
            return;
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            parts_ = parts;
            remaining_ = (int)th_.size();
            gen_++;
        }
        cv_.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [&]() { return remaining_ == 0; });
        job_ = nullptr;
    }

  private:
    void worker(int id) {
        uint64_t seen = 0;
        for (;;) {
            const std::function<void(int)>* j = nullptr;
            int parts = 0;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&]() { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                j = job_;
                parts = parts_;
            }
            if (id < parts) (*j)(id);
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (--remaining_ == 0) done_.notify_all();
            }
        }
    }
    int size_;
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int)>* job_ = nullptr;
    int parts_ = 0, remaining_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

// f(r0, r1) over row ranges, on the pool's workers.
template <class F>
void parallel_rows(int64_t rows, Pool& pool, F f) {
    const int64_t per_min = 16;
    const int p = (int)std::max<int64_t>(1, std::min<int64_t>(pool.size(), rows / per_min));
    pool.run(p, [&](int i) { f(rows * i / p, rows * (i + 1) / p); });
}

// Block of a matrix at nested quadrant indices (q_1 .. q_d), outer level
// first: its first row and first word.
struct BlockRef {
    int64_t row, word;
};

// Quadrant tuples of d levels (4^d, tuple index = q_1 * 4^(d-1) + ... + q_d)
// and their block offsets in a rows x words matrix.
std::vector<BlockRef> block_refs(int d, int64_t rows, int64_t words) {
    int64_t nt = 1;
    for (int l = 0; l < d; l++) nt *= 4;
    std::vector<BlockRef> v(nt);
    for (int64_t t = 0; t < nt; t++) {
        int64_t r = 0, w = 0, x = t;
        for (int l = d; l >= 1; l--) {  // digit of level l (innermost last)
            const int q = (int)(x % 4);
            x /= 4;
            r += (int64_t)(q >> 1) * (rows >> l);
            w += (int64_t)(q & 1) * (words >> l);
        }
        v[t] = {r, w};
    }
    return v;
}

// Digits (h_1 .. h_d) of sub-instance h, outer level first.
void digits7(int64_t h, int d, int* dig) {
    for (int l = d - 1; l >= 0; l--) {
        dig[l] = (int)(h % 7);
        h /= 7;
    }
}

// Tuples whose product of level masks is 1: sum of X blocks into out
// (Eq. igen, one sub-instance).
void generate(const uint64_t* X, int64_t rows, int64_t words, int d, const uint32_t* mask,
              const int* dig, const std::vector<BlockRef>& refs, uint64_t* out, Pool& pool) {
    std::vector<BlockRef> src;
    for (size_t t = 0; t < refs.size(); t++) {
        bool on = true;
        int64_t x = (int64_t)t;
        for (int l = d - 1; l >= 0 && on; l--) {
            const int q = (int)(x % 4);
            x /= 4;
            on = (mask[dig[l]] >> q) & 1u;
        }
        if (on) src.push_back(refs[t]);
    }
    const int64_t sr = rows >> d, sw = words >> d;
    parallel_rows(sr, pool, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; i++) {
            uint64_t* dst = out + i * sw;
            const uint64_t* s0 = X + (src[0].row + i) * words + src[0].word;
            std::memcpy(dst, s0, (size_t)sw * 8);
            for (size_t j = 1; j < src.size(); j++) {
                const uint64_t* sj = X + (src[j].row + i) * words + src[j].word;
                for (int64_t w = 0; w < sw; w++) dst[w] ^= sj[w];
            }
        }
    });
}

// Q_h into every C block whose zeta product is 1 (Eq. iagg), in one pass
// over Q's rows; a block's first contribution is copied, later ones added.
void aggregate(uint64_t* C, int64_t rows, int64_t words, int d, const uint32_t* zeta,
               const int* dig, const std::vector<BlockRef>& refs, std::vector<char>& seen,
               const uint64_t* Q, Pool& pool) {
    const int64_t sr = rows >> d, sw = words >> d;
    std::vector<BlockRef> dst;
    std::vector<char> first;
    for (size_t t = 0; t < refs.size(); t++) {
        bool on = true;
        int64_t x = (int64_t)t;
        for (int l = d - 1; l >= 0 && on; l--) {
            const int q = (int)(x % 4);
            x /= 4;
            on = (zeta[q] >> dig[l]) & 1u;
        }
        if (!on) continue;
        dst.push_back(refs[t]);
        first.push_back(!seen[t]);
        seen[t] = 1;
    }
    parallel_rows(sr, pool, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; i++) {
            const uint64_t* q = Q + i * sw;
            for (size_t j = 0; j < dst.size(); j++) {
                uint64_t* c = C + (dst[j].row + i) * words + dst[j].word;
                if (first[j])
                    std::memcpy(c, q, (size_t)sw * 8);
                else
                    for (int64_t w = 0; w < sw; w++) c[w] ^= q[w];
            }
        }
    });
}

// ---------------------------------------------------------------- device side
// Buffers kept between host-memory products on a device: pinning hundreds
// of MB of staging and allocating GBs of device memory cost tens of ms, a
// large share of one product. A call holds its device's cache (mutex),
// grows what it needs and leaves it for the next call;
// bmm_host_release frees it.
struct Cached {
    void* p = nullptr;
    uint64_t bytes = 0;
    bool pinned = false;
    bmm_status want(uint64_t b) {
        if (b <= bytes) return BMM_OK;
        release();
        const cudaError_t e = pinned ? cudaHostAlloc(&p, b, cudaHostAllocDefault) : cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return cuda_fail(e);
        }
        bytes = b;
        return BMM_OK;
    }
    void release() {
        if (p) {
            if (pinned)
                cudaFreeHost(p);
            else
                cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    uint64_t* w() const { return (uint64_t*)p; }
};

struct HostCache {
    std::mutex mu;
    // device: [0, 2) left operand slots, [2, 4) right, [4, 6) product, 6 scratch
    Cached dev[7];
    // pinned staging: [0, 2) T, [2, 4) S, [4, 6) Q
    Cached host[6];
    HostCache() {
        for (auto& h : host) h.pinned = true;
    }
    uint64_t device_bytes() const {
        uint64_t b = 0;
        for (const auto& d : dev) b += d.bytes;
        return b;
    }
    void release() {
        for (auto& d : dev) d.release();
        for (auto& h : host) h.release();
    }
};

constexpr int MAX_DEVICES = 64;
HostCache g_cache[MAX_DEVICES];

struct Streams {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev[12] = {nullptr};
    ~Streams() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
    }
    bmm_status make() {
        BMM_CUDA_TRY(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
        BMM_CUDA_TRY(cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking));
        for (auto& e : ev) BMM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return BMM_OK;
    }
};

// Device plans by shape (ragged edge blocks have their own).
struct PlanCache {
    int op;
    bmm_opts o;
    std::map<std::tuple<int64_t, int64_t, int64_t>, Plan> plans;
    bmm_status get(int64_t m, int64_t k, int64_t n, const Plan** out) {
        const auto key = std::make_tuple(m, k, n);
        auto it = plans.find(key);
        if (it == plans.end()) {
            Plan p;
            bmm_status st = make_plan(op, m, k, n, &o, &p);
            if (st != BMM_OK) return st;
            it = plans.emplace(key, p).first;
        }
        *out = &it->second;
        return BMM_OK;
    }
};

// Blocks of C, each with full k, streamed from and to the caller's arrays.
bmm_status run_blocked(const HostPlan& hp, const bmm_host_opts& ho, const uint64_t* A,
                       const uint64_t* B, uint64_t* C, cudaStream_t comp, HostCache& hc) {
    const int64_t m = hp.m, k = hp.k, n = hp.n, bm = hp.bm, bn = hp.bn;
    const int64_t kw = k / 64, nw = n / 64;
    const int64_t rm = (m + bm - 1) / bm, rn = (n + bn - 1) / bn;
    PlanCache pc{hp.op, ho.device, {}};
    pc.o.workspace = nullptr;
    pc.o.workspace_bytes = 0;
    Cached* dA = hc.dev;
    Cached* dB = hc.dev + 2;
    Cached* dC = hc.dev + 4;
    Cached& ws = hc.dev[6];
    for (int i = 0; i < 2; i++) {
        bmm_status st = dA[i].want((uint64_t)bm * k / 8);
        if (st == BMM_OK) st = dB[i].want((uint64_t)k * bn / 8);
        if (st == BMM_OK) st = dC[i].want((uint64_t)bm * bn / 8);
        if (st != BMM_OK) return st;
    }
    uint64_t wsb = 0;
    for (int64_t i = 0; i < rm; i++)
        for (int64_t j = 0; j < rn; j++) {
            const Plan* pl = nullptr;
            bmm_status st = pc.get(std::min(bm, m - i * bm), k, std::min(bn, n - j * bn), &pl);
            if (st != BMM_OK) return st;
            wsb = std::max(wsb, pl->workspace_bytes);
        }
    bmm_status st = ws.want(wsb);
    if (st != BMM_OK) return st;
    Streams sx;
    if ((st = sx.make()) != BMM_OK) return st;
    cudaEvent_t* a_up = sx.ev;       // [2] row panel of A uploaded
    cudaEvent_t* b_up = sx.ev + 2;   // [2] column panel of B uploaded
    cudaEvent_t* done = sx.ev + 4;   // [2] block product finished (its panels are free)
    cudaEvent_t* c_out = sx.ev + 6;  // [2] C block downloaded (its buffer is free)
    cudaEvent_t a_free[2] = {sx.ev[8], sx.ev[9]};  // last product of a row panel done
    int64_t t = 0;
    for (int64_t i = 0; i < rm; i++) {
        const int64_t mi = std::min(bm, m - i * bm);
        const int ai = (int)(i & 1);
        if (i >= 2) BMM_CUDA_TRY(cudaStreamWaitEvent(sx.up, a_free[ai], 0));
        BMM_CUDA_TRY(cudaMemcpyAsync(dA[ai].p, A + i * bm * kw, (size_t)mi * kw * 8,
                                     cudaMemcpyHostToDevice, sx.up));
        BMM_CUDA_TRY(cudaEventRecord(a_up[ai], sx.up));
        for (int64_t j = 0; j < rn; j++, t++) {
            const int64_t nj = std::min(bn, n - j * bn);
            const int bi = (int)(t & 1);
            if (t >= 2) BMM_CUDA_TRY(cudaStreamWaitEvent(sx.up, done[bi], 0));
            BMM_CUDA_TRY(cudaMemcpy2DAsync(dB[bi].p, (size_t)(nj / 64) * 8, B + j * (bn / 64),
                                           (size_t)nw * 8, (size_t)(nj / 64) * 8, (size_t)k,
                                           cudaMemcpyHostToDevice, sx.up));
            BMM_CUDA_TRY(cudaEventRecord(b_up[bi], sx.up));
            BMM_CUDA_TRY(cudaStreamWaitEvent(comp, a_up[ai], 0));
            BMM_CUDA_TRY(cudaStreamWaitEvent(comp, b_up[bi], 0));
            if (t >= 2) BMM_CUDA_TRY(cudaStreamWaitEvent(comp, c_out[bi], 0));
            const Plan* pl = nullptr;
            if ((st = pc.get(mi, k, nj, &pl)) != BMM_OK) return st;
            if ((st = execute_plan(*pl, dA[ai].w(), dB[bi].w(), dC[bi].w(), ws.p, comp)) !=
                BMM_OK)
                return st;
            BMM_CUDA_TRY(cudaEventRecord(done[bi], comp));
            if (j + 1 == rn) BMM_CUDA_TRY(cudaEventRecord(a_free[ai], comp));
            BMM_CUDA_TRY(cudaStreamWaitEvent(sx.down, done[bi], 0));
            BMM_CUDA_TRY(cudaMemcpy2DAsync(C + i * bm * nw + j * (bn / 64), (size_t)nw * 8,
                                           dC[bi].p, (size_t)(nj / 64) * 8,
                                           (size_t)(nj / 64) * 8, (size_t)mi,
                                           cudaMemcpyDeviceToHost, sx.down));
            BMM_CUDA_TRY(cudaEventRecord(c_out[bi], sx.down));
        }
    }
    BMM_CUDA_TRY(cudaStreamSynchronize(sx.down));
    BMM_CUDA_TRY(cudaStreamSynchronize(comp));
    return BMM_OK;
}

// Pipeline state of one double-buffered slot, shared by the three host roles.
struct Slots {
    std::mutex mu;
    std::condition_variable cv;
    int64_t generated[2] = {-1, -1};   // sub-instance whose T/S sit in the staging slot
    int64_t uploaded[2] = {-1, -1};    // sub-instance whose upload has been issued
    int64_t downloaded[2] = {-1, -1};  // sub-instance whose download has been issued
    int64_t aggregated[2] = {-1, -1};  // sub-instance folded into C (Q slot free again)
    bool failed = false;
    template <class P>
    bool wait(P pred) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&]() { return failed || pred(); });
        return !failed;
    }
    template <class F>
    void update(F f) {
        {
            std::lock_guard<std::mutex> lk(mu);
            f();
        }
        cv.notify_all();
    }
};

bmm_status run_host_strassen(const HostPlan& hp, const bmm_host_opts& ho, const uint64_t* A,
                             const uint64_t* B, uint64_t* C, cudaStream_t comp, HostCache& hc) {
    const int d = hp.host_depth;
    const int64_t m = hp.m, k = hp.k, n = hp.n;
    const int64_t sm = m >> d, sk = k >> d, sn = n >> d;
    const uint64_t tb = (uint64_t)sm * sk / 8, sb = (uint64_t)sk * sn / 8, qb = (uint64_t)sm * sn / 8;
    const int64_t count = hp.count;
    uint32_t xi[7], eta[7], zeta[4];
    switch (ho.device.variant) {
        case 0: slp::level_masks<0>(xi, eta, zeta); break;
        case 1: slp::level_masks<1>(xi, eta, zeta); break;
        default: slp::level_masks<2>(xi, eta, zeta); break;
    }
    PlanCache pc{hp.op, ho.device, {}};
    pc.o.workspace = nullptr;
    pc.o.workspace_bytes = 0;
    Cached* dT = hc.dev;
    Cached* dS = hc.dev + 2;
    Cached* dQ = hc.dev + 4;
    Cached& ws = hc.dev[6];
    Cached* hT = hc.host;
    Cached* hS = hc.host + 2;
    Cached* hQ = hc.host + 4;
    bmm_status st = BMM_OK;
    for (int i = 0; i < 2 && st == BMM_OK; i++) {
        st = dT[i].want(tb);
        if (st == BMM_OK) st = dS[i].want(sb);
        if (st == BMM_OK) st = dQ[i].want(qb);
        if (st == BMM_OK) st = hT[i].want(tb);
        if (st == BMM_OK) st = hS[i].want(sb);
        if (st == BMM_OK) st = hQ[i].want(qb);
    }
    if (st != BMM_OK) return st;
    const Plan* pl = nullptr;
    if ((st = pc.get(sm, sk, sn, &pl)) != BMM_OK) return st;
    if ((st = ws.want(pl->workspace_bytes)) != BMM_OK) return st;
    Streams sx;
    if ((st = sx.make()) != BMM_OK) return st;
    cudaEvent_t* up_done = sx.ev;    // [2] T/S of the slot uploaded (staging free)
    cudaEvent_t* comp_done = sx.ev + 2;  // [2] product of the slot finished
    cudaEvent_t* down_done = sx.ev + 4;  // [2] Q of the slot downloaded
    int dev = 0;
    cudaGetDevice(&dev);
    // generation and aggregation of neighbouring sub-instances overlap in
    // time, and each is memory-bound: both get every thread
    const int threads = host_threads(ho);
    const int gen_threads = threads, agg_threads = threads;
    const std::vector<BlockRef> refA = block_refs(d, m, k / 64);
    const std::vector<BlockRef> refB = block_refs(d, k, n / 64);
    const std::vector<BlockRef> refC = block_refs(d, m, n / 64);
    std::vector<char> seen(refC.size(), 0);
    Slots sl;
    bmm_status gen_st = BMM_OK, agg_st = BMM_OK;

    std::thread generator([&]() {
        cudaSetDevice(dev);
        Pool pool(gen_threads);
        for (int64_t h = 0; h < count; h++) {
            const int g = (int)(h & 1);
            // the slot's previous sub-instance must have left for the device
            if (!sl.wait([&]() { return sl.uploaded[g] >= h - 2; })) return;
            if (h >= 2 && cudaEventSynchronize(up_done[g]) != cudaSuccess) {
                gen_st = BMM_ERR_CUDA;
                sl.update([&]() { sl.failed = true; });
                return;
            }
            int dig[8];
            digits7(h, d, dig);
            generate(A, m, k / 64, d, xi, dig, refA, hT[g].w(), pool);
            generate(B, k, n / 64, d, eta, dig, refB, hS[g].w(), pool);
            sl.update([&]() { sl.generated[g] = h; });
        }
    });
    std::thread aggregator([&]() {
        cudaSetDevice(dev);
        Pool pool(agg_threads);
        for (int64_t h = 0; h < count; h++) {
            const int g = (int)(h & 1);
            if (!sl.wait([&]() { return sl.downloaded[g] >= h; })) return;
            if (cudaEventSynchronize(down_done[g]) != cudaSuccess) {
                agg_st = BMM_ERR_CUDA;
                sl.update([&]() { sl.failed = true; });
                return;
            }
            int dig[8];
            digits7(h, d, dig);
            aggregate(C, m, n / 64, d, zeta, dig, refC, seen, hQ[g].w(), pool);
            sl.update([&]() { sl.aggregated[g] = h; });
        }
    });

    auto fail = [&](bmm_status s) {
        sl.update([&]() { sl.failed = true; });
        return s;
    };
    for (int64_t h = 0; h < count && st == BMM_OK; h++) {
        const int g = (int)(h & 1);
        if (!sl.wait([&]() { return sl.generated[g] >= h; })) break;
        // device T/S of the slot: free once the product two back finished
        cudaError_t e = cudaSuccess;
        if (h >= 2) e = cudaStreamWaitEvent(sx.up, comp_done[g], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dT[g].p, hT[g].p, tb, cudaMemcpyHostToDevice, sx.up);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dS[g].p, hS[g].p, sb, cudaMemcpyHostToDevice, sx.up);
        if (e == cudaSuccess) e = cudaEventRecord(up_done[g], sx.up);
        if (e != cudaSuccess) {
            st = fail(cuda_fail(e));
            break;
        }
        sl.update([&]() { sl.uploaded[g] = h; });
        e = cudaStreamWaitEvent(comp, up_done[g], 0);
        if (e == cudaSuccess && h >= 2) e = cudaStreamWaitEvent(comp, down_done[g], 0);
        if (e != cudaSuccess) {
            st = fail(cuda_fail(e));
            break;
        }
        if ((st = execute_plan(*pl, dT[g].w(), dS[g].w(), dQ[g].w(), ws.p, comp)) != BMM_OK) {
            fail(st);
            break;
        }
        e = cudaEventRecord(comp_done[g], comp);
        // the pinned Q slot must have been folded into C
        if (e == cudaSuccess && !sl.wait([&]() { return sl.aggregated[g] >= h - 2; })) break;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sx.down, comp_done[g], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hQ[g].p, dQ[g].p, qb, cudaMemcpyDeviceToHost, sx.down);
        if (e == cudaSuccess) e = cudaEventRecord(down_done[g], sx.down);
        if (e != cudaSuccess) {
            st = fail(cuda_fail(e));
            break;
        }
        sl.update([&]() { sl.downloaded[g] = h; });
    }
    generator.join();
    aggregator.join();
    if (st == BMM_OK) st = gen_st != BMM_OK ? gen_st : agg_st;
    if (st == BMM_OK && sl.failed) st = BMM_ERR_CUDA;
    const cudaError_t e1 = cudaStreamSynchronize(comp);
    const cudaError_t e2 = cudaStreamSynchronize(sx.down);
    if (st == BMM_OK && e1 != cudaSuccess) st = cuda_fail(e1);
    if (st == BMM_OK && e2 != cudaSuccess) st = cuda_fail(e2);
    return st;
}

bmm_status check_host_args(int op, const uint64_t* A, const uint64_t* B, const uint64_t* C,
                           int64_t m, int64_t k, int64_t n, const bmm_host_opts* opts) {
    if (op != OP_GF2 && op != OP_BOOL) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    if (opts && (opts->host_depth < -1 || opts->threads < 0)) return BMM_ERR_INVALID;
    if (opts && opts->host_depth > 0 && op != OP_GF2) return BMM_ERR_INVALID;  // no additive inverse
    if (!A || !B || !C) return BMM_ERR_INVALID;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15u) return BMM_ERR_ALIGN;
    const uint64_t ab = (uint64_t)m * k / 8, bb = (uint64_t)k * n / 8, cb = (uint64_t)m * n / 8;
    auto over = [](const void* x, uint64_t xb, const void* y, uint64_t yb) {
        const uintptr_t a = (uintptr_t)x, b = (uintptr_t)y;
        return a < b + yb && b < a + xb;
    };
    if (over(C, cb, A, ab) || over(C, cb, B, bb)) return BMM_ERR_INVALID;
    return BMM_OK;
}

// cached: device bytes this device's cache already holds (usable again)
bmm_status budget_of(const bmm_host_opts& ho, uint64_t cached, uint64_t* budget) {
    if (ho.device_bytes) {
        *budget = ho.device_bytes;
        return BMM_OK;
    }
    size_t fr = 0, tot = 0;
    BMM_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    *budget = (uint64_t)((fr + cached) * 0.8);
    return BMM_OK;
}

HostCache* device_cache() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES) return nullptr;
    return &g_cache[d];
}

bmm_status host_product(int op, const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m,
                        int64_t k, int64_t n, const bmm_host_opts* opts, cudaStream_t s) {
    bmm_status st = check_host_args(op, A, B, C, m, k, n, opts);
    if (st != BMM_OK) return st;
    bmm_host_opts ho;
    bmm_host_opts_default(&ho);
    if (opts) ho = *opts;
    HostCache* hc = device_cache();
    if (!hc) return BMM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(hc->mu);
    uint64_t budget = 0;
    if ((st = budget_of(ho, hc->device_bytes(), &budget)) != BMM_OK) return st;
    HostPlan hp;
    if ((st = host_plan(op, m, k, n, ho, budget, &hp)) != BMM_OK) return st;
    // a larger plan than the cache holds: release first, so that the old and
    // the new buffers never coexist against the budget
    if (hc->device_bytes() > 0 && hp.device_bytes > hc->device_bytes()) hc->release();
    return hp.host_depth > 0 ? run_host_strassen(hp, ho, A, B, C, s, *hc)
                             : run_blocked(hp, ho, A, B, C, s, *hc);
}

}  // namespace
}  // namespace bmm

using namespace bmm;

extern "C" {

void bmm_host_opts_default(bmm_host_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    bmm_opts_default(&o->device);
    o->device_bytes = 0;
    o->host_depth = -1;
    o->threads = 0;
}

bmm_status bmm_host_plan(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_host_opts* opts,
                         bmm_host_plan_info* info) {
    if (!info || (op != OP_GF2 && op != OP_BOOL)) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    if (opts && (opts->host_depth < -1 || opts->threads < 0)) return BMM_ERR_INVALID;
    bmm_host_opts ho;
    bmm_host_opts_default(&ho);
    if (opts) ho = *opts;
    uint64_t budget = 0;
    bmm_status st = budget_of(ho, 0, &budget);
    if (st != BMM_OK) return st;
    HostPlan hp;
    if ((st = host_plan(op, m, k, n, ho, budget, &hp)) != BMM_OK) return st;
    info->host_depth = hp.host_depth;
    info->sub_m = hp.bm;
    info->sub_k = k >> hp.host_depth;
    info->sub_n = hp.bn;
    info->count = hp.count;
    info->device_bytes = hp.device_bytes;
    info->staging_bytes = hp.staging_bytes;
    info->upload_bytes = hp.upload_bytes;
    info->download_bytes = hp.download_bytes;
    return BMM_OK;
}

void bmm_host_release(void) {
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < MAX_DEVICES; d++) {
        std::lock_guard<std::mutex> lk(g_cache[d].mu);
        if (g_cache[d].device_bytes() == 0 && !g_cache[d].host[0].p) continue;
        cudaSetDevice(d);
        g_cache[d].release();
    }
    cudaSetDevice(cur);
}

bmm_status bmm_gf2_host(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                        int64_t n, const bmm_host_opts* opts, bmm_stream_t stream) {
    return host_product(OP_GF2, A, B, C, m, k, n, opts, (cudaStream_t)stream);
}

bmm_status bmm_bool_host(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                         int64_t n, const bmm_host_opts* opts, bmm_stream_t stream) {
    return host_product(OP_BOOL, A, B, C, m, k, n, opts, (cudaStream_t)stream);
}

}  // extern "C"
