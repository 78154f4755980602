// Serving: continuous batching of decode requests on one GPU.
//
// A request is F frames of one code (any q, N, channel, prior, schedule).
// The server owns one device pool of a fixed HBM budget.  A worker thread
// runs rounds: it admits queued requests (in arrival order) whose footprint —
// message workspace, observations, outputs and state — fits in the pool's
// free space, sets up their state on the device, and then launches one
// persistent kernel per schedule over the frames of every resident request,
// each frame advancing by at most `round_iters` iterations from where it
// stopped (its messages stay resident between rounds).  Frames that stop
// (H x = z or max_iter, Sec. 2) are retired after the round: their outputs
// are copied to the caller's host buffers, their pool space is freed and
// their waiters are woken.  Requests that arrive while others run are
// admitted at the next round boundary and share its launches.
//
// Two lanes, each with its own stream, launch tables and state buffers: light
// requests run in rounds the worker waits for; heavy requests (an iteration
// costing at least kHeavyUnits GF(16), N = 1000 frame-iterations) run in
// rounds on their own stream that the worker only polls between light rounds.
// A round lasts as long as its slowest frame, so without the split every light
// request would wait for round_iters iterations of the heaviest resident
// frame.  Requests are set up on a third stream (their pageable copies may
// wait for it), and a lane's stream waits for the setups before each round.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gfbp_internal.cuh"

namespace gfbp {
void set_error(const std::string& msg);
}

using namespace gfbp;
using Clock = std::chrono::steady_clock;

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) of the pool (host bookkeeping only).
class PoolAlloc {
  public:
    explicit PoolAlloc(size_t size) { free_[0] = size; }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Req {
    uint64_t id = 0;
    const gfbp_code* code = nullptr;
    int F = 0, schedule = 0, max_iter = 0, obs_stride = 0;
    std::vector<float> obs, fparam;
    gfbp_channel ch{};
    bool markov = false;
    std::vector<double> T;
    std::vector<int32_t> src_pos;
    int K = 0;
    uint8_t* hx = nullptr;
    int32_t* hit = nullptr;
    uint8_t* hconv = nullptr;
    // device placement
    size_t off = 0, bytes = 0, ws_bytes = 0;
    size_t o_obs = 0, o_fp = 0, o_state = 0, o_x = 0, o_it = 0, o_cv = 0, o_ws = 0;
    DecodeArgs A{};
    int state = 0;  // 0 queued, 1 resident, 2 done, 3 failed
    gfbp_status status = GFBP_OK;
    int rounds = 0;
    int lane = 0;   // 0 light, 1 heavy
    Clock::time_point t_submit, t_admit, t_done;
};

struct LaunchBufs {  // device tables of one round's mixed launch
    void* dmem = nullptr;
    int cap = 0;
    MixedLaunch m;
};

// One lane of rounds (see above).  `resident` is guarded by the server mutex;
// the rest belongs to the worker thread.
struct Lane {
    cudaStream_t stream = nullptr;
    LaunchBufs bufs[2];
    int* d_states = nullptr;   // the round's frame states, gathered (device)
    int* h_states = nullptr;   // and read back in one copy (pinned host)
    int states_cap = 0;
    std::vector<Req*> resident;
    std::vector<Req*> order[2];   // the round in flight: SUS, PUS requests in launch order
    cudaEvent_t done = nullptr;   // recorded after the round's state copy
    bool in_flight = false;
    bool wide = false;   // 512-thread CTAs for the lane-group level kernels (heavy lane)
};

constexpr double kHeavyUnits = 8.0;

}  // namespace

struct gfbp_server {
    size_t budget = 0;
    int round_iters = 8;
    void* pool = nullptr;
    cudaStream_t setup_stream = nullptr;
    cudaEvent_t setup_done = nullptr;   // recorded after each batch of setups
    std::unique_ptr<PoolAlloc> alloc;
    Lane lane[2];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    bool admit_blocked = false;   // the queue's head did not fit; cleared when space is freed
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    bool stop = false, draining = false;
    std::thread worker;
    int device = 0;
    // statistics
    long long rounds = 0, completed = 0;
    int peak_resident = 0;
    size_t peak_bytes = 0;
    uint32_t field_poly[8] = {0};
};

namespace {

size_t footprint(const Req& r, size_t* ws_out) {
    size_t ws = 0;
    gfbp_prior pr{};
    if (r.markov) { pr.kind = GFBP_PRIOR_MARKOV; pr.T = r.T.data(); pr.K = r.K; pr.src_pos = r.src_pos.data(); }
    gfbp_workspace_size(r.code, r.F, (gfbp_schedule)r.schedule, r.markov ? &pr : nullptr, 0, &ws);
    *ws_out = ws;
    const size_t N = (size_t)r.code->dev.N;
    return a256(ws) + a256(r.obs.size() * 4) + a256(r.fparam.size() * 4) + a256((size_t)r.F * 4) +
           a256((size_t)r.F * N) + a256((size_t)r.F * 4) + a256((size_t)r.F);
}

// The check-node route the server runs a code on (AUTO's choice).
int served_method(const CodeDev& c) { return c.q <= kAutoDirectMaxQ ? kDirect : kTransform; }

// Work of one iteration of one frame of this code in units of a GF(16),
// N = 1000 frame's iteration: edge-vector entries times the check node's work
// per entry (q for the probability route, 4 log2 q for the transforms).
double iteration_units(const CodeDev& c) {
    int lg = 0;
    while ((1 << lg) < c.q) lg++;
    const double work = (double)c.E * c.q * (served_method(c) == kDirect ? (double)c.q : 4.0 * lg);
    return work / (3000.0 * 16 * 16);
}

// Iterations a frame advances in one round.  Heavy lane: round_iters.  Light
// lane: round_iters for frames costing at most one unit, proportionally fewer
// for costlier ones (at least one), so that a light round lasts about
// round_iters unit iterations.
int round_iters_for(const Req& r, int round_iters) {
    if (r.lane == 1) return round_iters;
    const double n = round_iters / std::max(iteration_units(r.code->dev), 1e-9);
    return n >= round_iters ? round_iters : (n < 1.0 ? 1 : (int)n);
}

// Put an admitted request on the device: inputs, state, channel likelihoods
// and initial messages.  Runs on the worker thread, on the setup stream.
gfbp_status setup(gfbp_server* S, Req& r) {
    cudaStream_t st = S->setup_stream;
    uint8_t* base = static_cast<uint8_t*>(S->pool) + r.off;
    const size_t N = (size_t)r.code->dev.N;
    size_t o = 0;
    r.o_ws = o; o += a256(r.ws_bytes);
    r.o_obs = o; o += a256(r.obs.size() * 4);
    r.o_fp = o; o += a256(r.fparam.size() * 4);
    r.o_state = o; o += a256((size_t)r.F * 4);
    r.o_x = o; o += a256((size_t)r.F * N);
    r.o_it = o; o += a256((size_t)r.F * 4);
    r.o_cv = o;
    cudaError_t e = cudaMemcpyAsync(base + r.o_obs, r.obs.data(), r.obs.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !r.fparam.empty())
        e = cudaMemcpyAsync(base + r.o_fp, r.fparam.data(), r.fparam.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + r.o_state, 0, (size_t)r.F * 4, st);
    if (e != cudaSuccess) return GFBP_ECUDA;
    gfbp_channel ch = r.ch;
    ch.frame_param = r.fparam.empty() ? nullptr : reinterpret_cast<const float*>(base + r.o_fp);
    gfbp_prior pr{};
    if (r.markov) { pr.kind = GFBP_PRIOR_MARKOV; pr.T = r.T.data(); pr.K = r.K; pr.src_pos = r.src_pos.data(); }
    const int method = served_method(r.code->dev);
    e = batch_prepare_item(r.A, base + r.o_ws, r.code, r.F, reinterpret_cast<const float*>(base + r.o_obs), ch,
                           (gfbp_schedule)r.schedule, r.markov ? &pr : nullptr, r.max_iter, base + r.o_x,
                           reinterpret_cast<int32_t*>(base + r.o_it), base + r.o_cv, nullptr, method, nullptr,
                           st);
    if (e != cudaSuccess) return GFBP_EINVAL;
    r.A.fstate = reinterpret_cast<int*>(base + r.o_state);
    r.A.round_iters = round_iters_for(r, S->round_iters);
    e = launch_channel(r.A, st);
    if (e == cudaSuccess && r.A.markov) e = launch_fill_prior(r.A, st);
    if (e == cudaSuccess && r.schedule == GFBP_SUS) e = launch_init_dev(r.A, st);
    return e == cudaSuccess ? GFBP_OK : GFBP_ECUDA;
}

// Frame states of a round's launch in its frame-table order (item it's frames
// at prefix[it] ..), written at out, so that the host reads every resident
// frame's state in one copy instead of one per request.
__global__ void k_gather_states(const DecodeArgs* __restrict__ items, const int* __restrict__ prefix, int n_items,
                                int total, int* __restrict__ out) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_items - 1;   // the item whose frames hold g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        out[g] = items[lo].fstate[g - prefix[lo]];
    }
}

// Build and launch one schedule's mixed kernel over a lane's requests on its
// stream; `order` receives them in the launch's item order.
cudaError_t launch_round(Lane& L, int schedule, const std::vector<Req*>& rs, std::vector<Req*>* order) {
    std::vector<DecodeArgs> items;
    std::vector<int> prefix(1, 0), variant;
    int owner[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    std::vector<Req*> sel;
    std::vector<const CodeDev*> cd;
    for (Req* r : rs) {
        if (r->schedule != schedule) continue;
        sel.push_back(r);
        cd.push_back(&r->code->dev);
    }
    order->clear();
    for (int i : heavy_first(cd)) {
        Req* r = sel[i];
        order->push_back(r);
        const int pf = r->code->dev.p - 1;
        if (owner[pf] < 0) owner[pf] = (int)items.size();
        items.push_back(r->A);
        prefix.push_back(prefix.back() + r->F);
        variant.push_back(tuned_variant(r->code, schedule));
    }
    if (items.empty()) return cudaSuccess;
    LaunchBufs& B = L.bufs[schedule];
    const int n = (int)items.size();
    if (n > B.cap) {
        if (B.dmem) cudaFree(B.dmem);
        B.dmem = nullptr;
        const int cap = std::max(n, 2 * B.cap);
        const size_t cargs = a256(sizeof(DecodeArgs) * (size_t)cap), cint = a256(sizeof(int) * (size_t)(cap + 1));
        cudaError_t e = cudaMalloc(&B.dmem, cargs + 2 * cint + 512);
        if (e != cudaSuccess) { B.cap = 0; B.dmem = nullptr; return e; }
        B.cap = cap;
    }
    const size_t cargs = a256(sizeof(DecodeArgs) * (size_t)B.cap), cint = a256(sizeof(int) * (size_t)(B.cap + 1));
    uint8_t* base = static_cast<uint8_t*>(B.dmem);
    MixedLaunch& m = B.m;
    m.d_args = reinterpret_cast<DecodeArgs*>(base);
    m.d_prefix = reinterpret_cast<int*>(base + cargs);
    m.d_variant = reinterpret_cast<int*>(base + cargs + cint);
    m.d_counter = reinterpret_cast<int*>(base + cargs + 2 * cint);
    m.d_field = reinterpret_cast<int*>(base + cargs + 2 * cint + 256);
    m.n_items = n;
    m.total = prefix.back();
    m.schedule = schedule;
    m.wide = L.wide;
    cudaError_t e = cudaMemcpyAsync(m.d_args, items.data(), sizeof(DecodeArgs) * n, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.d_prefix, prefix.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.d_variant, variant.data(), sizeof(int) * n, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.d_field, owner, sizeof(owner), cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    mixed_shape(m, variant.data());
    return mixed_launch(m, L.stream);
}

// Start a round of a lane over `round` (its resident requests): the launches of
// both schedules after the setups recorded so far, the frame states gathered in
// launch order and copied back in one copy, then the lane's event.
cudaError_t start_round(gfbp_server* S, Lane& L, const std::vector<Req*>& round) {
    cudaError_t e = cudaStreamWaitEvent(L.stream, S->setup_done, 0);
    if (e == cudaSuccess) e = launch_round(L, GFBP_SUS, round, &L.order[0]);
    if (e == cudaSuccess) e = launch_round(L, GFBP_PUS, round, &L.order[1]);
    int total = 0;
    for (int k = 0; k < 2; k++)
        for (Req* r : L.order[k]) total += r->F;
    if (e == cudaSuccess && total > L.states_cap) {
        const int cap = std::max(total, 2 * L.states_cap + 1024);
        if (L.d_states) cudaFree(L.d_states);
        if (L.h_states) cudaFreeHost(L.h_states);
        L.d_states = nullptr;
        L.h_states = nullptr;
        L.states_cap = 0;
        e = cudaMalloc(&L.d_states, sizeof(int) * (size_t)cap);
        if (e == cudaSuccess) e = cudaMallocHost(&L.h_states, sizeof(int) * (size_t)cap);
        if (e == cudaSuccess) L.states_cap = cap;
    }
    int at = 0;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        const MixedLaunch& m = L.bufs[k == 0 ? GFBP_SUS : GFBP_PUS].m;
        int n = 0;
        for (Req* r : L.order[k]) n += r->F;
        if (n == 0) continue;
        const int blocks = std::min((n + 255) / 256, 1024);
        k_gather_states<<<blocks, 256, 0, L.stream>>>(m.d_args, m.d_prefix, m.n_items, n, L.d_states + at);
        e = cudaGetLastError();
        at += n;
    }
    if (e == cudaSuccess && total > 0)
        e = cudaMemcpyAsync(L.h_states, L.d_states, sizeof(int) * (size_t)total, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, L.stream);
    L.in_flight = e == cudaSuccess;
    return e;
}

// After a lane's round completed (e: its status): retire the requests whose
// frames have all stopped — outputs copied to their host buffers, pool space
// freed (the lane's stream has finished with it), waiters woken.
void finish_round(gfbp_server* S, Lane& L, cudaError_t e) {
    L.in_flight = false;
    std::vector<Req*> done;
    int at = 0;
    for (int k = 0; k < 2; k++) {
        for (Req* r : L.order[k]) {
            r->rounds++;
            bool all = e == cudaSuccess;
            for (int f = 0; f < r->F && all; f++) all = (L.h_states[at + f] >> 30) != 0;
            at += r->F;
            if (all || e != cudaSuccess) done.push_back(r);
        }
        L.order[k].clear();
    }
    for (Req* r : done) {
        const uint8_t* base = static_cast<const uint8_t*>(S->pool) + r->off;
        const size_t N = (size_t)r->code->dev.N;
        if (e == cudaSuccess) {
            cudaMemcpyAsync(r->hx, base + r->o_x, (size_t)r->F * N, cudaMemcpyDeviceToHost, L.stream);
            cudaMemcpyAsync(r->hit, base + r->o_it, (size_t)r->F * 4, cudaMemcpyDeviceToHost, L.stream);
            cudaMemcpyAsync(r->hconv, base + r->o_cv, (size_t)r->F, cudaMemcpyDeviceToHost, L.stream);
        }
    }
    if (!done.empty()) cudaStreamSynchronize(L.stream);
    std::lock_guard<std::mutex> lk(S->mu);
    S->rounds++;
    for (Req* r : done) {
        r->state = e == cudaSuccess ? 2 : 3;
        r->status = e == cudaSuccess ? GFBP_OK : GFBP_ECUDA;
        r->t_done = Clock::now();
        S->alloc->release(r->off, r->bytes);
        L.resident.erase(std::find(L.resident.begin(), L.resident.end(), r));
        S->completed++;
    }
    if (!done.empty()) {
        S->admit_blocked = false;
        S->cv_done.notify_all();
    }
}

bool lanes_idle(const gfbp_server* S) {
    return S->lane[0].resident.empty() && S->lane[1].resident.empty() && !S->lane[1].in_flight;
}

void worker_main(gfbp_server* S) {
    cudaSetDevice(S->device);
    Lane& light = S->lane[0];
    Lane& heavy = S->lane[1];
    for (;;) {
        std::vector<Req*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // with a heavy round in flight, poll it every millisecond
            S->cv_work.wait_for(lk, std::chrono::milliseconds(heavy.in_flight ? 1 : 20), [&] {
                return S->stop || (!S->queue.empty() && !S->admit_blocked) || !light.resident.empty() ||
                       (!heavy.resident.empty() && !heavy.in_flight);
            });
            if (S->stop && S->queue.empty() && lanes_idle(S)) break;
            // admission in arrival order while the footprint fits
            while (!S->queue.empty()) {
                Req* r = S->queue.front();
                size_t off = 0;
                if (!S->alloc->alloc(r->bytes, &off)) {
                    S->admit_blocked = true;
                    break;
                }
                S->queue.pop_front();
                r->off = off;
                r->t_admit = Clock::now();
                admitted.push_back(r);
            }
        }
        std::vector<Req*> failed;
        for (Req* r : admitted) {
            r->status = setup(S, *r);
            if (r->status != GFBP_OK) failed.push_back(r);
        }
        if (!admitted.empty()) cudaEventRecord(S->setup_done, S->setup_stream);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Req* r : admitted)
                if (r->status == GFBP_OK) {
                    r->state = 1;
                    S->lane[r->lane].resident.push_back(r);
                }
            S->peak_resident = std::max(S->peak_resident, (int)(light.resident.size() + heavy.resident.size()));
            S->peak_bytes = std::max(S->peak_bytes, S->alloc->used());
        }
        if (!failed.empty()) cudaStreamSynchronize(S->setup_stream);   // nothing of theirs in flight
        for (Req* r : failed) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->alloc->release(r->off, r->bytes);
            S->admit_blocked = false;
            r->state = 3;
            r->t_done = Clock::now();
            S->cv_done.notify_all();
        }
        // heavy lane: collect a finished round, start the next
        if (heavy.in_flight) {
            const cudaError_t q = cudaEventQuery(heavy.done);
            if (q != cudaErrorNotReady) finish_round(S, heavy, q);
        }
        if (!heavy.in_flight) {
            std::vector<Req*> round;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                round = heavy.resident;
            }
            if (!round.empty()) {
                const cudaError_t e = start_round(S, heavy, round);
                if (e != cudaSuccess) finish_round(S, heavy, e);
            }
        }
        // light lane: one round, waited for
        std::vector<Req*> round;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            round = light.resident;
        }
        if (!round.empty()) {
            cudaError_t e = start_round(S, light, round);
            if (e == cudaSuccess) e = cudaEventSynchronize(light.done);
            finish_round(S, light, e);
        }
    }
}

}  // namespace

extern "C" gfbp_status gfbp_server_create(size_t hbm_budget_bytes, int32_t round_iters, gfbp_server** out) {
    if (!out || hbm_budget_bytes < (1u << 20) || round_iters < 1) {
        set_error("gfbp_server_create: need a budget >= 1 MiB, round_iters >= 1 and an output handle");
        return GFBP_EINVAL;
    }
    *out = nullptr;
    gfbp_server* S = new (std::nothrow) gfbp_server();
    if (!S) { set_error("gfbp_server_create: out of host memory"); return GFBP_ENOMEM; }
    S->budget = hbm_budget_bytes;
    S->round_iters = round_iters;
    S->lane[1].wide = true;
    cudaGetDevice(&S->device);
    cudaError_t e = cudaMalloc(&S->pool, hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->setup_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->setup_done, cudaEventDisableTiming);
    for (Lane& L : S->lane) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_server_create: ") + cudaGetErrorString(e));
        for (Lane& L : S->lane) {
            if (L.done) cudaEventDestroy(L.done);
            if (L.stream) cudaStreamDestroy(L.stream);
        }
        if (S->setup_done) cudaEventDestroy(S->setup_done);
        if (S->setup_stream) cudaStreamDestroy(S->setup_stream);
        if (S->pool) cudaFree(S->pool);
        delete S;
        return e == cudaErrorMemoryAllocation ? GFBP_ENOMEM : GFBP_ECUDA;
    }
    S->alloc.reset(new PoolAlloc(hbm_budget_bytes));
    S->worker = std::thread(worker_main, S);
    *out = S;
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_server_submit(gfbp_server* S, const gfbp_request* q, uint64_t* id) {
    if (!S || !q || !id || !q->code || q->n_frames < 1 || !q->obs || !q->x_hat || !q->iters || !q->converged ||
        q->max_iter < 1 || (q->schedule != GFBP_PUS && q->schedule != GFBP_SUS)) {
        set_error("gfbp_server_submit: bad request");
        return GFBP_EINVAL;
    }
    const gfbp_code* c = q->code;
    if (c->dev.dcmax > 6 || c->dev.dvmax > 3) {
        set_error("gfbp_server_submit: served codes take row degree <= 6 and column degree <= 3");
        return GFBP_EUNSUPPORTED;
    }
    std::unique_ptr<Req> r(new Req());
    r->code = c;
    r->F = q->n_frames;
    r->schedule = q->schedule;
    r->max_iter = q->max_iter;
    r->ch = q->channel;
    const int p = c->dev.p, Qn = c->dev.q;
    const size_t per = q->channel.kind == GFBP_LOGLIK ? (size_t)Qn : (size_t)p;
    r->obs.assign(q->obs, q->obs + (size_t)q->n_frames * c->dev.N * per);
    if (q->channel.frame_param) r->fparam.assign(q->channel.frame_param, q->channel.frame_param + q->n_frames);
    r->ch.frame_param = nullptr;
    if (q->prior && q->prior->kind == GFBP_PRIOR_MARKOV) {
        if (!q->prior->T || q->prior->K < 1 || q->prior->K > c->dev.N) {
            set_error("gfbp_server_submit: Markov prior needs T and 1 <= K <= N");
            return GFBP_EINVAL;
        }
        r->markov = true;
        r->T.assign(q->prior->T, q->prior->T + (size_t)Qn * Qn);
        r->K = q->prior->K;
        r->src_pos.resize(r->K);
        for (int i = 0; i < r->K; i++) r->src_pos[i] = q->prior->src_pos ? q->prior->src_pos[i] : i;
    }
    r->hx = q->x_hat;
    r->hit = q->iters;
    r->hconv = q->converged;
    r->lane = iteration_units(c->dev) >= kHeavyUnits ? 1 : 0;
    r->bytes = footprint(*r, &r->ws_bytes);
    if (r->bytes > S->budget) {
        set_error("gfbp_server_submit: the request's device footprint (" + std::to_string(r->bytes) +
                  " bytes) exceeds the server budget");
        return GFBP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->draining || S->stop) {
        set_error("gfbp_server_submit: the server is draining");
        return GFBP_EBUSY;
    }
    const int pf = p - 1;
    if (S->field_poly[pf] && S->field_poly[pf] != c->poly) {
        set_error("gfbp_server_submit: codes of the same field size must use the same field polynomial");
        return GFBP_EUNSUPPORTED;
    }
    S->field_poly[pf] = c->poly;
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    *id = r->id;
    S->queue.push_back(r.get());
    S->reqs[r->id] = std::move(r);
    S->cv_work.notify_one();
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_server_wait(gfbp_server* S, uint64_t id, int64_t timeout_us, gfbp_result* res) {
    if (!S) { set_error("gfbp_server_wait: NULL server"); return GFBP_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) { set_error("gfbp_server_wait: unknown request id"); return GFBP_EINVAL; }
    Req* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (r->state < 2) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2) {
            set_error("gfbp_server_wait: timed out");
            return GFBP_ETIMEOUT;
        }
    }
    if (res) {
        res->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
        res->queue_us = std::chrono::duration<double, std::micro>(r->t_admit - r->t_submit).count();
        res->rounds = r->rounds;
    }
    const gfbp_status st = r->state == 2 ? GFBP_OK : r->status;
    S->reqs.erase(it);
    if (st != GFBP_OK) set_error("gfbp_server_wait: the request failed on the device");
    return st;
}

extern "C" gfbp_status gfbp_server_stats(gfbp_server* S, gfbp_server_stats_t* out) {
    if (!S || !out) { set_error("gfbp_server_stats: NULL argument"); return GFBP_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int32_t)S->queue.size();
    out->resident = (int32_t)(S->lane[0].resident.size() + S->lane[1].resident.size());
    out->peak_resident = S->peak_resident;
    out->rounds = S->rounds;
    out->completed = S->completed;
    out->bytes_in_use = S->alloc->used();
    out->peak_bytes = S->peak_bytes;
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_server_drain(gfbp_server* S) {
    if (!S) { set_error("gfbp_server_drain: NULL server"); return GFBP_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    S->draining = true;
    S->cv_work.notify_one();
    while (!S->queue.empty() || !S->lane[0].resident.empty() || !S->lane[1].resident.empty())
        S->cv_done.wait_for(lk, std::chrono::milliseconds(20));
    return GFBP_OK;
}

extern "C" void gfbp_server_destroy(gfbp_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->draining = true;
    }
    S->cv_work.notify_one();
    if (S->worker.joinable()) S->worker.join();
    for (Lane& L : S->lane) {
        for (auto& b : L.bufs)
            if (b.dmem) cudaFree(b.dmem);
        if (L.d_states) cudaFree(L.d_states);
        if (L.h_states) cudaFreeHost(L.h_states);
        cudaEventDestroy(L.done);
        cudaStreamDestroy(L.stream);
    }
    cudaEventDestroy(S->setup_done);
    cudaStreamDestroy(S->setup_stream);
    cudaFree(S->pool);
    delete S;
}
