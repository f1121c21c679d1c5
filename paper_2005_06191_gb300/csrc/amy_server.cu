// amy_server.cu -- request loop with continuous batching (the serving side of
// the C ABI: amy_server_create / amy_submit / amy_poll / amy_wait / amy_cancel).
//
// A scheduler thread owns one CUDA stream.  Each loop iteration it
//   1. drops cancelled requests,
//   2. admits queued requests in arrival order while a slot is free and the
//      device-memory budget allows: one stream-ordered allocation holds the
//      problem's geometry, parameters, per-dimension tables, V ping-pong pair,
//      mask and outputs; the tables and V_N are built on the device;
//   3. runs one tick: every resident problem advances one backup -- all in one
//      persistent batched kernel when the problem fits it, otherwise one
//      launch per problem -- and problems whose last backup ran copy V_0 and
//      pi_0 out, free their memory and publish their result.
// Requests arriving while others run join at the next tick (continuous
// batching).  Every problem's arithmetic is that of a single amy_synthesize
// call with the separable stored mode, so results do not depend on the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/amy.h"
#include "amy_fast.cuh"
#include "amy_internal.h"

using namespace amy;

namespace {

double now_us() {
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

enum ReqState { RQ_QUEUED = 0, RQ_RESIDENT = 1, RQ_DONE = 2 };

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

struct Req {
    uint64_t ticket = 0;
    Geom g;
    std::vector<double> params;
    std::vector<int32_t> upart;
    int64_t tab_words = 0;
    SpecDev spec;
    int32_t prec = AMY_PREC_FP32, v_store = AMY_V_NATIVE, horizon = 0;
    int state = RQ_QUEUED;
    bool cancel = false;
    amy_status status = AMY_OK;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    std::vector<float> V;
    std::vector<uint16_t> pi;
    // resident state (scheduler thread only)
    size_t dbytes = 0;
    void *dmem = nullptr;
    Geom *d_geom = nullptr;
    void *d_V[2] = {nullptr, nullptr};
    uint8_t *d_mask = nullptr;
    uint32_t *d_tab = nullptr;
    float *d_T = nullptr;      // factored rows: masses [sum W][pairs]
    int16_t *d_O = nullptr;    // factored rows: origins [n][pairs]
    float *d_Vout = nullptr;
    uint16_t *d_pi = nullptr;
    int cur = 0;
    int32_t k_left = 0;
    int tm = TM_SEPARABLE;  // row mode: separable tables, factored per-pair rows, or on the fly
    int wm = 0;
    int var = 0;  // fast-kernel variant (general / exact widths / exact + contiguous row)
    bool batched = false;
    int ulanes = 1;
    int64_t ntiles = 0;
    bool finishing = false;
    char *h_up = nullptr;   // pinned upload staging (geometry, parameters, table index parts)
    size_t h_up_bytes = 0;
    char *h_out = nullptr;  // pinned copy-out staging (V_0 then pi_0)
    size_t h_out_bytes = 0;
    cudaEvent_t done_ev = nullptr;
};

size_t vbytes(const Req *r) { return r->v_store == AMY_V_NATIVE ? 4 : 2; }

size_t npairs_of(const Req *r) { return (size_t)r->g.nx * (size_t)r->g.nu; }

size_t device_bytes(const Req *r) {
    const size_t nx = (size_t)r->g.nx;
    const size_t tab = r->tm == TM_SEPARABLE ? (size_t)r->tab_words * 4 : 0;
    const size_t fT = r->tm == TM_FACTORED ? npairs_of(r) * r->g.wsum * 4 : 0;
    const size_t fO = r->tm == TM_FACTORED ? npairs_of(r) * r->g.n * 2 : 0;
    return align256(sizeof(Geom)) + align256(r->params.size() * 8) + align256(tab) + align256(fT) + align256(fO) +
           2 * align256((nx + 2 * kVGuard) * vbytes(r)) + align256(nx) + align256(nx * 4) + align256(nx * 2);
}

}  // namespace

// Pinned host buffers reused across requests (uploads and copy-outs), so
// that every host<->device copy of the scheduler is asynchronous.
struct PinnedPool {
    std::map<size_t, std::vector<void *>> free_by_size;
    std::vector<void *> all;
    static size_t cls(size_t b) {
        size_t c = 4096;
        while (c < b) c <<= 1;
        return c;
    }
    void *get(size_t bytes) {
        const size_t c = cls(bytes);
        auto &v = free_by_size[c];
        if (!v.empty()) {
            void *p = v.back();
            v.pop_back();
            return p;
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, c) != cudaSuccess) return nullptr;
        all.push_back(p);
        return p;
    }
    void put(void *p, size_t bytes) {
        if (p) free_by_size[cls(bytes)].push_back(p);
    }
    void release_all() {
        for (void *p : all) cudaFreeHost(p);
        all.clear();
        free_by_size.clear();
    }
};

constexpr int kTickRing = 8;  // ticks the scheduler may run ahead of the GPU

constexpr int kMaxGroups = 64;  // kernel variants per tick (storage x width x mode x exact)

struct TickSlot {
    BatchEntry *h = nullptr;
    BatchEntry *d = nullptr;
    int32_t *counter = nullptr;  // one tile counter per group
    cudaEvent_t ev = nullptr;
    bool used = false;
};

struct amy_server_s {
    amy_server_opts opts;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_init;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Req *> resident;  // scheduler thread only: taking part in ticks
    std::deque<Req *> draining;   // scheduler thread only: copy-out (or cancel) enqueued, not yet published
    uint64_t next_ticket = 1;
    int64_t bytes_in_use = 0;
    int64_t in_flight = 0;  // queued + resident + draining
    bool stop = false;
    bool init_done = false;
    amy_status init_status = AMY_OK;
    std::string init_err;
    cudaStream_t stream = nullptr;
    // the requests' device memory: a pool of the server's own that keeps
    // freed memory mapped up to the budget (the device's default pool hands
    // it back to the driver at every synchronisation, and the next admission
    // pays for mapping it again)
    cudaMemPool_t pool = nullptr;
    int sm_count = 0;
    TickSlot ring[kTickRing];
    int64_t tick_no = 0;
    PinnedPool pinned;
    std::vector<cudaEvent_t> ev_pool;
    std::atomic<int64_t> completed{0}, ticks{0}, launches{0};
    std::atomic<int32_t> n_resident{0};
    std::map<std::string, int> tune;  // input lanes per shape class
    std::string tune_path;
    // CUDA graphs of tick layouts (opts.use_graphs): the tick's launches for a
    // given list of (resident problem, V parity), captured on the second
    // sighting of the layout and replayed while it repeats; each graph owns
    // the device copy of its batch tables and tile counters
    struct TickGraph {
        cudaGraphExec_t exec = nullptr;
        void *dmem = nullptr;  // batch tables + tile counters
        int64_t last_used = 0;
    };
    std::map<std::vector<uint64_t>, TickGraph> graphs;
    std::map<std::vector<uint64_t>, int64_t> layouts_seen;
    std::atomic<int64_t> graph_replays{0}, graph_captures{0};
};

namespace {

std::string shape_key(const Req *r, bool exact) {
    auto lg = [](int64_t v) {
        int b = 0;
        while ((1LL << (b + 1)) <= v) ++b;
        return b;
    };
    std::ostringstream o;
    o << r->g.n << "," << r->wm << "," << (exact ? 1 : 0) << "," << lg(r->g.nu) << "," << lg(r->g.nx) << ","
      << r->v_store << "," << r->tm;
    return o.str();
}

void load_tune(amy_server_s *s) {
    const char *p = std::getenv("AMY_AUTOTUNE_CACHE");
    if (!p || !*p) return;
    s->tune_path = p;
    std::ifstream f(p);
    std::string k;
    int ul;
    while (f >> k >> ul)
        if (ul == 1 || ul == 2 || ul == 4 || ul == 8) s->tune[k] = ul;
}

void save_tune(amy_server_s *s) {
    if (s->tune_path.empty()) return;
    std::ofstream f(s->tune_path);
    for (auto &kv : s->tune) f << kv.first << " " << kv.second << "\n";
}

cudaEvent_t get_event(amy_server_s *s) {
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

FastCall fast_call(const Req *r, const void *Vn, void *Vo, float *Vfinal, uint16_t *pi, int ulanes) {
    FastCall c;
    c.Vn = Vn;
    c.Vo = Vo;
    c.Vfinal = Vfinal;
    c.pi = pi;
    c.mask = r->d_mask;
    c.spec_kind = r->spec.kind;
    c.kahan = r->prec == AMY_PREC_FP32_KAHAN;
    c.T = r->d_T;
    c.O = r->d_O;
    c.npairs = (int64_t)npairs_of(r);
    c.tab = r->d_tab;
    c.ulanes = ulanes;
    c.grouped = r->tm == TM_SEPARABLE && input_runs_share_outer(r->g, r->upart);
    c.runs = c.grouped ? input_outer_runs(r->g, r->upart) : 0;
    return c;
}

// Autotuner: the input-lane count (threads per state) of the register-
// resident backup, chosen per shape class by timing each candidate on the
// first admitted problem of the class (writes only the scratch V vector).
amy_status autotune(amy_server_s *s, Req *r) {
    bool exact = true;
    for (int d = 0; d < r->g.n; ++d) exact = exact && r->g.W[d] == r->wm;
    const std::string key = shape_key(r, exact);
    auto it = s->tune.find(key);
    if (it != s->tune.end()) {
        r->ulanes = it->second;
        return AMY_OK;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return set_error(AMY_E_CUDA, "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return set_error(AMY_E_CUDA, "event");
    }
    float best = 1e30f;
    int best_ul = fast_default_ulanes(r->g, s->sm_count);
    for (int ul = 1; ul <= 8; ul <<= 1) {
        if (ul > 1 && ul > r->g.nu) break;
        FastCall c = fast_call(r, r->d_V[0], r->d_V[1], nullptr, nullptr, ul);
        amy_status st = launch_backup_fast(r->g, r->tm, r->v_store, c, s->sm_count, s->stream);
        if (st == AMY_OK) {
            cudaEventRecord(a, s->stream);
            for (int rep = 0; rep < 3 && st == AMY_OK; ++rep)
                st = launch_backup_fast(r->g, r->tm, r->v_store, c, s->sm_count, s->stream);
            cudaEventRecord(b, s->stream);
        }
        if (st != AMY_OK) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return st;
        }
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return cuda_error(e, "autotune timing");
        }
        s->launches += 4;
        if (ms < best) {
            best = ms;
            best_ul = ul;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    s->tune[key] = best_ul;
    r->ulanes = best_ul;
    return AMY_OK;
}

void carve(Req *r) {
    char *p = (char *)r->dmem;
    const size_t nx = (size_t)r->g.nx;
    r->d_geom = (Geom *)p;
    p += align256(sizeof(Geom));
    double *d_params = (double *)p;
    p += align256(r->params.size() * 8);
    r->d_tab = (uint32_t *)p;
    p += align256(r->tm == TM_SEPARABLE ? (size_t)r->tab_words * 4 : 0);
    r->d_T = (float *)p;
    p += align256(r->tm == TM_FACTORED ? npairs_of(r) * r->g.wsum * 4 : 0);
    r->d_O = (int16_t *)p;
    p += align256(r->tm == TM_FACTORED ? npairs_of(r) * r->g.n * 2 : 0);
    r->d_V[0] = p + kVGuard * vbytes(r);
    p += align256((nx + 2 * kVGuard) * vbytes(r));
    r->d_V[1] = p + kVGuard * vbytes(r);
    p += align256((nx + 2 * kVGuard) * vbytes(r));
    r->d_mask = (uint8_t *)p;
    p += align256(nx);
    r->d_Vout = (float *)p;
    p += align256(nx * 4);
    r->d_pi = (uint16_t *)p;
    r->g.params = d_params;
}

// Admission: device memory, uploads (through pinned staging), tables and V_N,
// all stream-ordered on the server stream; only the first problem of a new
// shape class waits (autotuning).
amy_status admit(amy_server_s *s, Req *r) {
    r->dbytes = device_bytes(r);
    cudaError_t e = cudaMallocFromPoolAsync(&r->dmem, r->dbytes, s->pool, s->stream);
    if (e != cudaSuccess) return cuda_error(e, "request memory");
    carve(r);
    // finite guard cells around both V buffers (read with zero mass)
    e = cudaMemsetAsync((char *)r->d_V[0] - kVGuard * vbytes(r), 0, align256((r->g.nx + 2 * kVGuard) * vbytes(r)) * 2,
                        s->stream);
    if (e != cudaSuccess) return cuda_error(e, "guard init");
    const size_t pbytes = r->params.size() * 8;
    const size_t ubytes = r->tm == TM_SEPARABLE ? r->upart.size() * 4 : 0;
    r->h_up_bytes = sizeof(Geom) + pbytes + ubytes;
    r->h_up = (char *)s->pinned.get(r->h_up_bytes);
    if (!r->h_up) return set_error(AMY_E_OUT_OF_MEMORY, "pinned staging");
    memcpy(r->h_up, &r->g, sizeof(Geom));
    memcpy(r->h_up + sizeof(Geom), r->params.data(), pbytes);
    if (ubytes) memcpy(r->h_up + sizeof(Geom) + pbytes, r->upart.data(), ubytes);
    e = cudaMemcpyAsync(r->d_geom, r->h_up, sizeof(Geom), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)r->g.params, r->h_up + sizeof(Geom), pbytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && ubytes)
        e = cudaMemcpyAsync(r->d_tab + r->g.uoff, r->h_up + sizeof(Geom) + pbytes, ubytes, cudaMemcpyHostToDevice,
                            s->stream);
    if (e != cudaSuccess) return cuda_error(e, "request upload");
    amy_status st = AMY_OK;
    if (r->tm == TM_SEPARABLE) {
        st = launch_build_sep(r->g, r->d_tab, s->sm_count, s->stream);
        s->launches += 1;
    } else if (r->tm == TM_FACTORED) {
        st = launch_build_factored(r->g, r->d_T, r->d_O, (int64_t)npairs_of(r), s->sm_count, s->stream);
        s->launches += 1;
    }
    if (st == AMY_OK) st = launch_spec_mask(r->g, r->spec, r->d_mask, r->d_V[0], r->v_store, s->stream);
    if (st != AMY_OK) return st;
    s->launches += 1;
    r->wm = fast_wm(r->g, AMY_PREC_FP32);
    r->var = r->wm > 0 ? fast_variant(r->g, r->wm, r->tm) : 0;
    r->batched = r->wm > 0 && batched_smem_bytes(r->g.n, r->wm) <= 100 * 1024;
    if (r->wm > 0) {
        st = autotune(s, r);
        if (st != AMY_OK) return st;
    }
    r->ntiles = ((int64_t)r->g.nx * r->ulanes + FAST_THREADS - 1) / FAST_THREADS;
    r->cur = 0;
    r->k_left = r->horizon;
    if (r->horizon == 0) {
        // V_0 = V_N; no policy entries
        if (r->v_store == AMY_V_NATIVE)
            e = cudaMemcpyAsync(r->d_Vout, r->d_V[0], (size_t)r->g.nx * 4, cudaMemcpyDeviceToDevice, s->stream);
        else
            st = launch_v16_to_f32(r->d_V[0], r->v_store, r->d_Vout, r->g.nx, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "V_N copy");
        if (st != AMY_OK) return st;
        e = cudaMemsetAsync(r->d_pi, 0xFF, (size_t)r->g.nx * 2, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "policy init");
        r->finishing = true;
    }
    return AMY_OK;
}

// Publishes a finished request (lock held by the caller).
void publish(amy_server_s *s, Req *r, amy_status st) {
    r->status = st;
    r->state = RQ_DONE;
    r->t_finish = now_us();
    s->in_flight -= 1;
    s->completed += 1;
    s->cv_done.notify_all();
}

void forget_graphs(amy_server_s *s, const Req *r);

// A resident request leaves the ticks: copy V_0 / pi_0 out (unless
// cancelled), free its device memory (stream-ordered) and record the event
// after which its result can be published.
amy_status retire(amy_server_s *s, Req *r, bool copy_out) {
    forget_graphs(s, r);
    cudaError_t e = cudaSuccess;
    if (copy_out) {
        r->h_out_bytes = (size_t)r->g.nx * 6;
        r->h_out = (char *)s->pinned.get(r->h_out_bytes);
        if (!r->h_out) return set_error(AMY_E_OUT_OF_MEMORY, "pinned staging");
        e = cudaMemcpyAsync(r->h_out, r->d_Vout, (size_t)r->g.nx * 4, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->h_out + (size_t)r->g.nx * 4, r->d_pi, (size_t)r->g.nx * 2, cudaMemcpyDeviceToHost,
                                s->stream);
    }
    if (e == cudaSuccess && r->dmem) e = cudaFreeAsync(r->dmem, s->stream);
    r->dmem = nullptr;
    r->done_ev = get_event(s);
    if (e == cudaSuccess && r->done_ev) e = cudaEventRecord(r->done_ev, s->stream);
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "retire");
}

// Publishes drained requests whose copy-out has completed (lock held).
// block = true waits for the oldest one.
void drain(amy_server_s *s, std::unique_lock<std::mutex> &lk, bool block) {
    while (!s->draining.empty()) {
        Req *r = s->draining.front();
        if (r->done_ev) {
            cudaError_t q = cudaEventQuery(r->done_ev);
            if (q == cudaErrorNotReady) {
                if (!block) return;
                lk.unlock();
                cudaEventSynchronize(r->done_ev);
                lk.lock();
                block = false;
                continue;
            }
        }
        s->draining.pop_front();
        amy_status st = r->cancel ? AMY_E_CANCELLED : r->status;
        if (st == AMY_OK && r->h_out) {
            r->V.resize(r->g.nx);
            r->pi.resize(r->g.nx);
            memcpy(r->V.data(), r->h_out, (size_t)r->g.nx * 4);
            memcpy(r->pi.data(), r->h_out + (size_t)r->g.nx * 4, (size_t)r->g.nx * 2);
        }
        s->pinned.put(r->h_out, r->h_out_bytes);
        s->pinned.put(r->h_up, r->h_up_bytes);
        r->h_out = r->h_up = nullptr;
        if (r->done_ev) s->ev_pool.push_back(r->done_ev);
        r->done_ev = nullptr;
        r->upart.clear();
        r->upart.shrink_to_fit();
        publish(s, r, st);
    }
}

constexpr size_t kMaxTickGraphs = 32;

void drop_graph(amy_server_s *s, amy_server_s::TickGraph &tg) {
    if (tg.exec) cudaGraphExecDestroy(tg.exec);
    if (tg.dmem) cudaFreeAsync(tg.dmem, s->stream);
    tg.exec = nullptr;
    tg.dmem = nullptr;
}

// Drops every tick graph (and layout count) whose layout contains r, when r
// leaves the resident set: its device memory is freed, and a later request
// may be allocated at the same host address.
void forget_graphs(amy_server_s *s, const Req *r) {
    const uint64_t tag = (uint64_t)(uintptr_t)r << 1;
    auto has = [&](const std::vector<uint64_t> &k) {
        for (uint64_t v : k)
            if ((v & ~1ull) == tag) return true;
        return false;
    };
    for (auto it = s->graphs.begin(); it != s->graphs.end();) {
        if (has(it->first)) {
            drop_graph(s, it->second);
            it = s->graphs.erase(it);
        } else {
            ++it;
        }
    }
    for (auto it = s->layouts_seen.begin(); it != s->layouts_seen.end();) {
        if (has(it->first))
            it = s->layouts_seen.erase(it);
        else
            ++it;
    }
}

amy_status tick_launches(amy_server_s *s, TickSlot &slot, bool graphs, bool capture,
                         const std::vector<uint64_t> &key);

// One tick: every resident problem advances one backup -- the batched ones in
// one persistent launch -- without waiting for the GPU (up to kTickRing ticks
// run ahead).  With opts.use_graphs the tick's launches are a CUDA graph of
// its layout (which problems take part, in which order, at which V parity),
// captured the second time the layout occurs and replayed while it repeats
// (a stable set of residents alternates between two layouts).  In that mode
// every tick writes V_k and pi_k to the problems' output buffers, so that the
// layout does not depend on which problems take their last step (the last
// tick's values are the ones copied out, as without graphs).
amy_status tick(amy_server_s *s) {
    TickSlot &slot = s->ring[s->tick_no % kTickRing];
    if (slot.used) {
        cudaError_t e = cudaEventSynchronize(slot.ev);
        if (e != cudaSuccess) return cuda_error(e, "tick slot");
    }
    const bool graphs = s->opts.use_graphs != 0;
    std::vector<uint64_t> key;
    amy_server_s::TickGraph *cached = nullptr;
    bool capture = false;
    if (graphs) {
        for (Req *r : s->resident)
            if (r->k_left > 0 && !r->finishing) key.push_back(((uint64_t)(uintptr_t)r << 1) | (uint64_t)r->cur);
        auto it = s->graphs.find(key);
        if (it != s->graphs.end()) {
            cached = &it->second;
        } else {
            capture = ++s->layouts_seen[key] >= 2;
            if (s->layouts_seen.size() > 4 * kMaxTickGraphs) s->layouts_seen.clear();
        }
    }
    if (cached) {
        cudaError_t e = cudaGraphLaunch(cached->exec, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "tick graph launch");
        cached->last_used = s->tick_no;
        s->graph_replays += 1;
        s->launches += 1;
    } else {
        amy_status st = tick_launches(s, slot, graphs, capture, key);
        if (st != AMY_OK) return st;
    }
    cudaError_t e = cudaEventRecord(slot.ev, s->stream);
    if (e != cudaSuccess) return cuda_error(e, "tick event");
    slot.used = true;
    s->tick_no += 1;
    for (Req *r : s->resident) {
        if (r->k_left <= 0 || r->finishing) continue;
        r->cur ^= 1;
        r->k_left -= 1;
        if (r->k_left == 0) r->finishing = true;
    }
    s->ticks += 1;
    return AMY_OK;
}

// The launches of one tick, enqueued directly (batch tables uploaded from the
// tick slot), or -- capture -- as a new graph of this layout: its batch
// tables are uploaded once into device memory the graph owns, the launches
// are captured and the graph is launched.
amy_status tick_launches(amy_server_s *s, TickSlot &slot, bool graphs, bool capture,
                         const std::vector<uint64_t> &key) {
    // group the batched problems by kernel variant; the rest launch one by one
    struct Group {
        int vt, wm, tm, var;
        std::vector<Req *> rs;
    };
    std::vector<Group> groups;
    std::vector<Req *> singles;
    for (Req *r : s->resident) {
        if (r->k_left <= 0 || r->finishing) continue;
        if (s->opts.batched && r->batched) {
            Group *gp = nullptr;
            for (Group &gg : groups)
                if (gg.vt == r->v_store && gg.wm == r->wm && gg.tm == r->tm && gg.var == r->var) gp = &gg;
            if (!gp) {
                groups.push_back({r->v_store, r->wm, r->tm, r->var, {}});
                gp = &groups.back();
            }
            gp->rs.push_back(r);
        } else {
            singles.push_back(r);
        }
    }
    // batch tables in the tick slot's pinned buffer; with a capture they go to
    // device memory of the graph's own, uploaded before the capture begins
    BatchEntry *d_tab = slot.d;
    int32_t *d_cnt = slot.counter;
    void *gmem = nullptr;
    int32_t ne = 0;
    for (size_t gi = 0; gi < groups.size() && gi < (size_t)kMaxGroups; ++gi)
        for (Req *r : groups[gi].rs) {
            (void)r;
            ++ne;
        }
    if (capture) {
        const size_t tb = align256(sizeof(BatchEntry) * (size_t)std::max(ne, 1));
        cudaError_t e = cudaMallocFromPoolAsync(&gmem, tb + sizeof(int32_t) * kMaxGroups, s->pool, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "tick graph tables");
        d_tab = (BatchEntry *)gmem;
        d_cnt = (int32_t *)((char *)gmem + tb);
    }
    ne = 0;
    std::vector<int32_t> gfirst, gcount;
    std::vector<int64_t> gtiles;
    std::vector<int> gmaxn;
    for (size_t gi = 0; gi < groups.size() && gi < (size_t)kMaxGroups; ++gi) {
        Group &gg = groups[gi];
        const int32_t first = ne;
        int64_t tiles = 0;
        int max_n = 1;
        for (Req *r : gg.rs) {
            const bool last = graphs || r->k_left == 1;
            BatchEntry &e = slot.h[ne++];
            e.g = r->d_geom;
            e.Vn = r->d_V[r->cur];
            e.Vo = r->d_V[r->cur ^ 1];
            e.Vfinal = last ? r->d_Vout : nullptr;
            e.pi = last ? r->d_pi : nullptr;
            e.mask = r->d_mask;
            e.tab = r->d_tab;
            e.T = r->d_T;
            e.O = r->d_O;
            e.npairs = (int64_t)npairs_of(r);
            e.tile_begin = tiles;
            e.tm = r->tm;
            e.spec_kind = r->spec.kind;
            e.kahan = r->prec == AMY_PREC_FP32_KAHAN;
            e.vt = r->v_store;
            e.wm = r->wm;
            e.ulanes = r->ulanes;
            e.tileX = FAST_THREADS / r->ulanes;
            tiles += r->ntiles;
            max_n = std::max(max_n, r->g.n);
        }
        gfirst.push_back(first);
        gcount.push_back(ne - first);
        gtiles.push_back(tiles);
        gmaxn.push_back(max_n);
    }
    if (ne > 0) {
        cudaError_t e = cudaMemcpyAsync(d_tab, slot.h, sizeof(BatchEntry) * ne, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) {
            if (gmem) cudaFreeAsync(gmem, s->stream);
            return cuda_error(e, "step table upload");
        }
    }
    if (capture) {
        cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaFreeAsync(gmem, s->stream);
            return cuda_error(e, "tick capture");
        }
    }
    amy_status st = AMY_OK;
    for (size_t gi = 0; gi < gfirst.size() && st == AMY_OK; ++gi) {
        const Group &gg = groups[gi];
        st = launch_step_group(gg.vt, gg.wm, gg.tm, gg.var, d_tab + gfirst[gi], gcount[gi], gtiles[gi], d_cnt + gi,
                               gmaxn[gi], s->sm_count, s->stream);
    }
    for (size_t i = 0; i < singles.size() && st == AMY_OK; ++i) {
        Req *r = singles[i];
        const bool last = graphs || r->k_left == 1;
        FastCall c = fast_call(r, r->d_V[r->cur], r->d_V[r->cur ^ 1], last ? r->d_Vout : nullptr,
                               last ? r->d_pi : nullptr, r->ulanes);
        st = r->wm > 0 ? launch_backup_fast(r->g, r->tm, r->v_store, c, s->sm_count, s->stream)
                       : launch_backup_generic_fp32(r->g, r->tm, c, r->v_store, s->sm_count, s->stream);
    }
    if (capture) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && st == AMY_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st == AMY_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, s->stream);
        if (st != AMY_OK || e != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            cudaFreeAsync(gmem, s->stream);
            return st != AMY_OK ? st : cuda_error(e, "tick graph");
        }
        // keep at most kMaxTickGraphs graphs: the least recently used goes
        if (s->graphs.size() >= kMaxTickGraphs) {
            auto lru = s->graphs.begin();
            for (auto it = s->graphs.begin(); it != s->graphs.end(); ++it)
                if (it->second.last_used < lru->second.last_used) lru = it;
            drop_graph(s, lru->second);
            s->graphs.erase(lru);
        }
        amy_server_s::TickGraph &tg = s->graphs[key];
        tg.exec = exec;
        tg.dmem = gmem;
        tg.last_used = s->tick_no;
        s->layouts_seen.erase(key);
        s->graph_captures += 1;
        s->launches += 1;
        return AMY_OK;
    }
    if (st != AMY_OK) return st;
    s->launches += (int64_t)gfirst.size() + (int64_t)singles.size();
    return AMY_OK;
}

void scheduler(amy_server_s *s) {
    cudaError_t e = cudaSetDevice(s->opts.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->opts.device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaMemPoolProps pp;
        std::memset(&pp, 0, sizeof pp);
        pp.allocType = cudaMemAllocationTypePinned;
        pp.handleTypes = cudaMemHandleTypeNone;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = s->opts.device;
        e = cudaMemPoolCreate(&s->pool, &pp);
        uint64_t keep = s->opts.device_mem_budget > 0 ? (uint64_t)s->opts.device_mem_budget : ~0ull;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int i = 0; i < kTickRing && e == cudaSuccess; ++i) {
        TickSlot &t = s->ring[i];
        e = cudaMallocHost(&t.h, sizeof(BatchEntry) * s->opts.max_slots);
        if (e == cudaSuccess) e = cudaMalloc(&t.d, sizeof(BatchEntry) * s->opts.max_slots);
        if (e == cudaSuccess) e = cudaMalloc(&t.counter, sizeof(int32_t) * kMaxGroups);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->init_done = true;
        if (e != cudaSuccess) {
            s->init_status = AMY_E_CUDA;
            s->init_err = cudaGetErrorString(e);
        }
        s->cv_init.notify_all();
    }
    if (e != cudaSuccess) return;
    std::unique_lock<std::mutex> lk(s->mu);
    auto fail_all = [&](amy_status st) {
        lk.unlock();
        cudaStreamSynchronize(s->stream);
        lk.lock();
        for (auto &kv : s->graphs) drop_graph(s, kv.second);
        s->graphs.clear();
        s->layouts_seen.clear();
        for (Req *r : s->resident) {
            if (r->dmem) cudaFreeAsync(r->dmem, s->stream);
            r->dmem = nullptr;
            s->bytes_in_use -= (int64_t)r->dbytes;
            r->status = st;
            s->draining.push_back(r);
        }
        s->resident.clear();
        for (Req *r : s->draining)
            if (r->status == AMY_OK) r->status = st;
    };
    while (true) {
        drain(s, lk, false);
        // cancelled residents leave at the tick boundary
        for (size_t i = 0; i < s->resident.size();) {
            Req *r = s->resident[i];
            if (r->cancel) {
                s->resident.erase(s->resident.begin() + i);
                s->bytes_in_use -= (int64_t)r->dbytes;
                if (retire(s, r, false) != AMY_OK) r->status = AMY_E_CUDA;
                s->draining.push_back(r);
            } else {
                ++i;
            }
        }
        if (s->stop) break;
        // admission in arrival order while a slot and memory are free
        while (!s->queue.empty() && (int)s->resident.size() < s->opts.max_slots) {
            Req *r = s->queue.front();
            if (r->cancel) {
                s->queue.pop_front();
                publish(s, r, AMY_E_CANCELLED);
                continue;
            }
            const int64_t need = (int64_t)device_bytes(r);
            if (s->bytes_in_use + need > s->opts.device_mem_budget) {
                if (!s->resident.empty() || !s->draining.empty()) break;  // wait for memory to free up
                s->queue.pop_front();                                      // can never fit
                publish(s, r, set_error(AMY_E_OUT_OF_MEMORY, "request exceeds the server memory budget"));
                continue;
            }
            s->queue.pop_front();
            r->state = RQ_RESIDENT;
            r->t_admit = now_us();
            s->bytes_in_use += need;
            lk.unlock();
            amy_status st = admit(s, r);
            lk.lock();
            if (st != AMY_OK) {
                if (r->dmem) cudaFreeAsync(r->dmem, s->stream);
                r->dmem = nullptr;
                s->bytes_in_use -= need;
                r->status = st;
                s->draining.push_back(r);
                continue;
            }
            s->resident.push_back(r);
        }
        s->n_resident = (int32_t)s->resident.size();
        bool active = false;
        for (Req *r : s->resident) active = active || (r->k_left > 0 && !r->finishing);
        bool any_finishing = false;
        for (Req *r : s->resident) any_finishing = any_finishing || r->finishing;
        if (!active && !any_finishing) {
            if (!s->draining.empty()) {
                drain(s, lk, true);
                continue;
            }
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            continue;
        }
        lk.unlock();
        amy_status st = active ? tick(s) : AMY_OK;
        lk.lock();
        if (st != AMY_OK) {
            fail_all(st);
            continue;
        }
        // problems whose last backup was enqueued copy out and leave
        for (size_t i = 0; i < s->resident.size();) {
            Req *r = s->resident[i];
            if (r->finishing) {
                s->resident.erase(s->resident.begin() + i);
                s->bytes_in_use -= (int64_t)r->dbytes;
                amy_status rs = retire(s, r, !r->cancel);
                if (rs != AMY_OK) r->status = rs;
                s->draining.push_back(r);
            } else {
                ++i;
            }
        }
    }
    // shutdown: everything still queued or resident is cancelled
    for (Req *r : s->resident) {
        r->cancel = true;
        retire(s, r, false);
        s->draining.push_back(r);
    }
    s->resident.clear();
    while (!s->queue.empty()) {
        publish(s, s->queue.front(), AMY_E_CANCELLED);
        s->queue.pop_front();
    }
    lk.unlock();
    cudaStreamSynchronize(s->stream);
    lk.lock();
    drain(s, lk, true);
}

amy_status fill_result(amy_server_s *s, Req *r, amy_result *out) {
    memset(out, 0, sizeof *out);
    out->status = r->status;
    out->n_states = r->g.nx;
    out->submit_us = r->t_submit;
    out->admit_us = r->t_admit;
    out->finish_us = r->t_finish;
    if (r->status == AMY_OK) {
        out->V = (float *)std::malloc(sizeof(float) * r->V.size());
        out->policy = (uint16_t *)std::malloc(sizeof(uint16_t) * r->pi.size());
        if (!out->V || !out->policy) {
            std::free(out->V);
            std::free(out->policy);
            memset(out, 0, sizeof *out);
            return set_error(AMY_E_OUT_OF_MEMORY, "result copy");
        }
        memcpy(out->V, r->V.data(), sizeof(float) * r->V.size());
        memcpy(out->policy, r->pi.data(), sizeof(uint16_t) * r->pi.size());
    }
    s->reqs.erase(r->ticket);
    delete r;
    return AMY_OK;
}

}  // namespace

extern "C" {

amy_status amy_server_create(const amy_server_opts *opts, amy_server *out) {
    if (!opts || !out) return set_error(AMY_E_INVALID_ARG, "null argument");
    *out = nullptr;
    amy_server_s *s = new (std::nothrow) amy_server_s();
    if (!s) return set_error(AMY_E_OUT_OF_MEMORY, "server allocation");
    s->opts = *opts;
    if (s->opts.device_mem_budget <= 0) s->opts.device_mem_budget = 4LL << 30;
    if (s->opts.max_slots <= 0) s->opts.max_slots = 64;
    if (s->opts.max_queue <= 0) s->opts.max_queue = 4096;
    load_tune(s);
    s->th = std::thread(scheduler, s);
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_init.wait(lk, [&] { return s->init_done; });
    if (s->init_status != AMY_OK) {
        const std::string msg = s->init_err;
        lk.unlock();
        s->th.join();
        delete s;
        return set_error(AMY_E_CUDA, "server init: %s", msg.c_str());
    }
    lk.unlock();
    *out = s;
    return AMY_OK;
}

amy_status amy_submit(amy_server s, const amy_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (req->prec != AMY_PREC_FP32 && req->prec != AMY_PREC_FP32_KAHAN)
        return set_error(AMY_E_UNSUPPORTED, "served requests run in FP32 or FP32_KAHAN");
    if (req->v_store < AMY_V_NATIVE || req->v_store > AMY_V_UNORM16) return set_error(AMY_E_INVALID_ARG, "bad v_store");
    if (req->horizon < 0) return set_error(AMY_E_INVALID_ARG, "negative horizon");
    Req *r = new (std::nothrow) Req();
    if (!r) return set_error(AMY_E_OUT_OF_MEMORY, "request allocation");
    amy_status st = make_geom(&req->sys, &req->states, &req->inputs, req->sigma, &req->cut, r->g, r->params);
    if (st == AMY_OK && r->g.sys == SYS_EXPR)
        st = set_error(AMY_E_UNSUPPORTED, "text systems are built with amy_build (their mean tables need a handle)");
    if (st == AMY_OK && r->g.noise == NOISE_USER)
        st = set_error(AMY_E_UNSUPPORTED, "user noise densities are built with amy_build (their tables need a handle)");
    if (st == AMY_OK) st = make_spec(r->g, &req->spec, r->spec);
    if (st == AMY_OK) st = plan_sep_tables(r->g, r->params, r->tab_words, &r->upart);
    if (st != AMY_OK) {
        delete r;
        return st;
    }
    // per-dimension tables only when they stay small (few dependencies);
    // otherwise rows are recomputed on the fly and need no memory
    // row mode: separable tables when small, per-pair factored rows when they
    // fit a quarter of the budget, otherwise on the fly (no row memory)
    r->tm = choose_tmode(r->g, r->params, req->prec, s->opts.device_mem_budget);
    if (r->tm != TM_SEPARABLE) {
        r->upart.clear();
        r->upart.shrink_to_fit();
    }
    r->prec = req->prec;
    r->v_store = req->v_store;
    r->horizon = req->horizon;
    r->t_submit = now_us();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->in_flight >= s->opts.max_queue) {
        delete r;
        return set_error(AMY_E_QUEUE_FULL, "server queue is full");
    }
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    s->in_flight += 1;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return AMY_OK;
}

amy_status amy_poll(amy_server s, uint64_t ticket, amy_result *out) {
    if (!s || !out) return set_error(AMY_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(AMY_E_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state != RQ_DONE) return AMY_E_NOT_READY;
    return fill_result(s, it->second, out);
}

amy_status amy_wait(amy_server s, uint64_t ticket, int64_t timeout_us, amy_result *out) {
    if (!s || !out) return set_error(AMY_E_INVALID_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(AMY_E_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *r = it->second;
    auto ready = [&] { return r->state == RQ_DONE; };
    if (timeout_us < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return set_error(AMY_E_TIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    }
    return fill_result(s, r, out);
}

amy_status amy_cancel(amy_server s, uint64_t ticket) {
    if (!s) return set_error(AMY_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(AMY_E_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *r = it->second;
    if (r->state == RQ_DONE) return AMY_OK;
    r->cancel = true;
    if (r->state == RQ_QUEUED) {
        auto q = std::find(s->queue.begin(), s->queue.end(), r);
        if (q != s->queue.end()) s->queue.erase(q);
        publish(s, r, AMY_E_CANCELLED);
    }
    return AMY_OK;
}

amy_status amy_server_stats(amy_server s, int64_t *completed, int64_t *ticks, int64_t *launches, int32_t *resident) {
    if (!s) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (completed) *completed = s->completed;
    if (ticks) *ticks = s->ticks;
    if (launches) *launches = s->launches;
    if (resident) *resident = s->n_resident;
    return AMY_OK;
}

amy_status amy_server_graph_stats(amy_server s, int64_t *captures, int64_t *replays) {
    if (!s) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (captures) *captures = s->graph_captures;
    if (replays) *replays = s->graph_replays;
    return AMY_OK;
}

void amy_server_destroy(amy_server s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    save_tune(s);
    for (auto &kv : s->graphs) drop_graph(s, kv.second);
    s->graphs.clear();
    for (auto &kv : s->reqs) delete kv.second;
    for (TickSlot &t : s->ring) {
        if (t.h) cudaFreeHost(t.h);
        cudaFree(t.d);
        cudaFree(t.counter);
        if (t.ev) cudaEventDestroy(t.ev);
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->pinned.release_all();
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

void amy_result_free(amy_result *r) {
    if (!r) return;
    std::free(r->V);
    std::free(r->policy);
    r->V = nullptr;
    r->policy = nullptr;
}

}  // extern "C"
