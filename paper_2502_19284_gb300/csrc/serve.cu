// Serving loop: requests (SpMV and PageRank iterations) on a resident set of converted
// matrices, admitted by free slots and free memory, with continuous batching.
//
// A worker thread owns every CUDA call.  Each admission scans the queue in arrival order:
// the first request that fits the memory budget opens a group; a SpMV group then takes every
// later queued SpMV request with the same vector type and accumulation (up to max_batch)
// that still fits, and runs them as one batched launch on a free slot's stream; a PageRank
// request runs alone (its iteration graph uses the matrix's own scratch, so at most one per
// matrix is in flight).  Slots run concurrently, so requests that arrive while others are on
// the GPU start as soon as a slot and memory free up.  Completion is detected by polling each
// slot's event; latency = completion - arrival on the host's steady clock.
//
// Results do not depend on the mix: a batched product is, per request, bitwise the
// single-vector merge product with the same accumulation, and PageRank is one fixed graph.
#include "common.cuh"
#include "convert.cuh"

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <string>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace spmv {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

spmv_status check(cudaError_t e, const char *what) { return e == cudaSuccess ? SPMV_OK : cuda_status(e, what); }

struct Req {
    spmv_request r;
    int64_t ticket = 0;
    double t_arr = 0, t_done = 0;
    int64_t bytes = 0;          // device bytes reserved against the budget
    void *dx = nullptr, *dy = nullptr;
    size_t xb = 0, yb = 0;      // bytes of x and y
    size_t stage_in = 0, stage_out = 0;   // offsets in the slot's pinned staging (pageable x / y)
    bool x_direct = false, y_direct = false;
    spmv_status st = SPMV_OK;
    std::string msg;            // error text recorded on the worker thread
    bool done = false;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    BatchSlot *bs = nullptr;
    bool busy = false;
    std::vector<Req *> reqs;
    int64_t bytes = 0;
    unsigned char *pin = nullptr;   // pinned staging for pageable inputs and outputs
    size_t pin_cap = 0;
};

struct Mat {
    spmv_matrix *h = nullptr;
    int64_t bytes = 0;
    bool pr_busy = false;
    double *pr_x = nullptr;         // PageRank output kept on the device (one captured graph)
};

bool is_device_or_pinned(const void *p, bool *device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        *device = false;
        return false;
    }
    *device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    return a.type != cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace spmv

struct spmv_server {
    spmv_server_opts o{};
    int device = 0;
    std::vector<spmv::Mat> mats;
    std::vector<spmv::Slot> slots;
    std::deque<spmv::Req *> queue;
    std::unordered_map<int64_t, spmv::Req *> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int64_t next_ticket = 1;
    int64_t resident = 0, inflight = 0;
    spmv_server_stats_t st{};
};

namespace spmv {
namespace {

int64_t request_bytes(const spmv_server *S, const Req *q) {
    const spmv_matrix *h = S->mats[q->r.matrix].h;
    if (q->r.kind == SPMV_REQ_PAGERANK) return 0;   // output and scratch belong to the matrix
    spmv_matrix *hs[1] = {const_cast<spmv_matrix *>(h)};
    return (int64_t)(round256(q->xb) + round256(q->yb)) + batch_scratch_bytes(1, hs, 1);
}

void finish_slot(spmv_server *S, Slot &sl, cudaError_t e) {
    const double t = now_s();
    for (Req *q : sl.reqs) {
        if (e != cudaSuccess && q->st == SPMV_OK) {
            q->st = cuda_status(e, "served request");
            q->msg = spmv_last_error();
        }
        if (q->st == SPMV_OK && !q->y_direct) {
            const void *src = q->r.kind == SPMV_REQ_PAGERANK ? (const void *)sl.pin : (const void *)(sl.pin + q->stage_out);
            std::memcpy(q->r.y, src, q->yb);
        }
        if (q->dx) dev_free_async(q->dx, sl.s);
        if (q->dy && q->r.kind == SPMV_REQ_SPMV) dev_free_async(q->dy, sl.s);
        q->dx = q->dy = nullptr;
        if (q->r.kind == SPMV_REQ_PAGERANK) S->mats[q->r.matrix].pr_busy = false;
        q->t_done = t;
        q->done = true;
        if (q->st == SPMV_OK) ++S->st.completed;
        else ++S->st.failed;
    }
    S->inflight -= sl.bytes;
    sl.bytes = 0;
    sl.busy = false;
    sl.reqs.clear();
    S->cv_done.notify_all();
}

spmv_status grow_pin(Slot &sl, size_t need) {
    if (need <= sl.pin_cap) return SPMV_OK;
    if (sl.pin) cudaFreeHost(sl.pin);
    sl.pin = nullptr;
    sl.pin_cap = 0;
    SPMV_CUDA_TRY(cudaHostAlloc((void **)&sl.pin, need, cudaHostAllocDefault));
    sl.pin_cap = need;
    return SPMV_OK;
}

// Enqueue one group on a free slot.  Errors are recorded on the requests; the slot's event
// is recorded in every case, so completion handling stays uniform.
void launch_group(spmv_server *S, Slot &sl, std::vector<Req *> &grp, int64_t bytes) {
    sl.busy = true;
    sl.reqs = grp;
    sl.bytes = bytes;
    S->inflight += bytes;
    S->st.peak_bytes = std::max<int64_t>(S->st.peak_bytes, S->resident + S->inflight);
    cudaStream_t s = sl.s;
    spmv_status st = SPMV_OK;
    Req *q0 = grp[0];
    if (q0->r.kind == SPMV_REQ_PAGERANK) {
        Mat &M = S->mats[q0->r.matrix];
        M.pr_busy = true;
        const int64_t n = M.h->n;
        if (!M.pr_x) {
            st = dev_alloc((void **)&M.pr_x, (size_t)std::max<int64_t>(n, 1) * 8, "served PageRank output", s);
            if (st == SPMV_OK) {
                const int64_t before = M.h->bytes;
                st = pagerank(M.h, q0->r.damping, q0->r.iters, M.pr_x, s);
                S->resident += (M.h->bytes - before) + n * 8;   // the matrix's PageRank scratch stays
            }
        } else {
            st = pagerank(M.h, q0->r.damping, q0->r.iters, M.pr_x, s);
        }
        if (st == SPMV_OK) {
            if (q0->y_direct) {
                st = check(cudaMemcpyAsync(q0->r.y, M.pr_x, q0->yb, cudaMemcpyDefault, s), "PageRank output");
            } else if ((st = grow_pin(sl, q0->yb)) == SPMV_OK) {
                st = check(cudaMemcpyAsync(sl.pin, M.pr_x, q0->yb, cudaMemcpyDeviceToHost, s), "PageRank output");
            }
        }
        q0->st = st;
    } else {
        size_t stage = 0;
        for (Req *q : grp) {
            q->stage_in = stage;
            if (!q->x_direct) stage += round256(q->xb);
            q->stage_out = stage;
            if (!q->y_direct) stage += round256(q->yb);
        }
        st = grow_pin(sl, std::max<size_t>(stage, 256));
        std::vector<spmv_matrix *> hs;
        std::vector<const void *> X;
        std::vector<void *> Y;
        for (Req *q : grp) {
            if (st != SPMV_OK) break;
            spmv_matrix *h = S->mats[q->r.matrix].h;
            bool dev = false;
            if (q->x_direct && is_device_or_pinned(q->r.x, &dev) && dev) {
                q->dx = nullptr;
                X.push_back(q->r.x);
            } else {
                if ((st = dev_alloc(&q->dx, std::max<size_t>(q->xb, 16), "served x", s)) != SPMV_OK) break;
                const void *src = q->r.x;
                if (!q->x_direct) {
                    std::memcpy(sl.pin + q->stage_in, q->r.x, q->xb);
                    src = sl.pin + q->stage_in;
                }
                if (q->xb && (st = check(cudaMemcpyAsync(q->dx, src, q->xb, cudaMemcpyDefault, s), "served x")) !=
                                 SPMV_OK)
                    break;
                X.push_back(q->dx);
            }
            if ((st = dev_alloc(&q->dy, std::max<size_t>(q->yb, 16), "served y", s)) != SPMV_OK) break;
            Y.push_back(q->dy);
            hs.push_back(h);
        }
        if (st == SPMV_OK)
            st = batch_direct(sl.bs, (int)hs.size(), hs.data(), 1, X.data(), Y.data(), (spmv_dtype)q0->r.vec_dt,
                              q0->r.accum, s);
        for (Req *q : grp) {
            if (st != SPMV_OK || !q->dy) break;
            void *dst = q->y_direct ? q->r.y : (void *)(sl.pin + q->stage_out);
            if (q->yb) st = check(cudaMemcpyAsync(dst, q->dy, q->yb, cudaMemcpyDefault, s), "served y");
        }
        for (Req *q : grp) q->st = st;
        ++S->st.launches;
        S->st.batched_requests += (int64_t)grp.size();
    }
    const cudaError_t e = cudaEventRecord(sl.ev, s);
    if (e != cudaSuccess)
        for (Req *q : grp)
            if (q->st == SPMV_OK) q->st = cuda_status(e, "served request event");
    for (Req *q : grp)
        if (q->st != SPMV_OK && q->msg.empty()) q->msg = spmv_last_error();
}

void admit(spmv_server *S) {
    for (;;) {
        Slot *free = nullptr;
        bool any_busy = false;
        for (Slot &sl : S->slots) {
            if (sl.busy) any_busy = true;
            else if (!free) free = &sl;
        }
        if (!free || S->queue.empty()) return;
        std::vector<Req *> grp;
        int64_t need = 0;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            Req *q = *it;
            Mat &M = S->mats[q->r.matrix];
            if (grp.empty()) {
                if (q->r.kind == SPMV_REQ_PAGERANK && M.pr_busy) {
                    ++it;
                    continue;
                }
                const int64_t b = q->bytes;
                if (S->resident + S->inflight + b > S->o.budget_bytes) {
                    if (!any_busy) {   // cannot fit even alone: fail it rather than wait forever
                        q->st = SPMV_ERR_OOM;
                        q->msg = "spmv_server: the request does not fit the memory budget even alone";
                        q->done = true;
                        q->t_done = now_s();
                        ++S->st.failed;
                        it = S->queue.erase(it);
                        S->cv_done.notify_all();
                        continue;
                    }
                    ++S->st.deferred;
                    break;
                }
                grp.push_back(q);
                need = b;
                it = S->queue.erase(it);
                if (q->r.kind == SPMV_REQ_PAGERANK) break;
            } else {
                const Req *g0 = grp[0];
                if (q->r.kind != SPMV_REQ_SPMV || (int)grp.size() >= S->o.max_batch || q->r.vec_dt != g0->r.vec_dt ||
                    q->r.accum != g0->r.accum || M.h->dt != S->mats[g0->r.matrix].h->dt ||
                    S->resident + S->inflight + need + q->bytes > S->o.budget_bytes) {
                    ++it;
                    continue;
                }
                grp.push_back(q);
                need += q->bytes;
                it = S->queue.erase(it);
            }
        }
        if (grp.empty()) return;
        launch_group(S, *free, grp, need);
    }
}

void worker_loop(spmv_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool busy = false;
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            finish_slot(S, sl, e);
        }
        admit(S);
        busy = false;
        for (Slot &sl : S->slots) busy = busy || sl.busy;
        if (S->stop && S->queue.empty() && !busy) break;
        if (!busy) {
            S->cv_work.wait(lk);
            continue;
        }
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
    }
}

spmv_status submit_at(spmv_server *S, const spmv_request *r, double t_arr, int64_t *ticket) {
    if (!r || r->matrix < 0 || (size_t)r->matrix >= S->mats.size() ||
        (r->kind != SPMV_REQ_SPMV && r->kind != SPMV_REQ_PAGERANK) || !r->y) {
        set_error("spmv_server_submit: bad request (kind, matrix id or output)");
        return SPMV_ERR_INVALID_ARG;
    }
    const spmv_matrix *h = S->mats[r->matrix].h;
    Req *q = new Req();
    q->r = *r;
    q->t_arr = t_arr;
    if (r->kind == SPMV_REQ_SPMV) {
        if ((r->vec_dt != SPMV_F64 && r->vec_dt != SPMV_F32) || (h->n > 0 && !r->x)) {
            delete q;
            set_error("spmv_server_submit: SpMV needs x and vec_dt SPMV_F64 or SPMV_F32");
            return SPMV_ERR_INVALID_ARG;
        }
        const size_t es = r->vec_dt == SPMV_F64 ? 8 : 4;
        q->xb = (size_t)h->n * es;
        q->yb = (size_t)h->m * es;
    } else {
        if (h->m != h->n || r->iters < 0 || r->iters > 10000 || !(r->damping >= 0.0 && r->damping <= 1.0)) {
            delete q;
            set_error("spmv_server_submit: PageRank needs a square matrix, 0 <= iters <= 10000, damping in [0, 1]");
            return SPMV_ERR_INVALID_ARG;
        }
        q->yb = (size_t)h->n * 8;
    }
    bool dev = false;
    q->x_direct = r->kind == SPMV_REQ_SPMV && r->x && is_device_or_pinned(r->x, &dev);
    q->y_direct = is_device_or_pinned(r->y, &dev);
    std::lock_guard<std::mutex> g(S->mu);
    q->bytes = request_bytes(S, q);
    q->ticket = S->next_ticket++;
    S->reqs[q->ticket] = q;
    S->queue.push_back(q);
    ++S->st.submitted;
    *ticket = q->ticket;
    S->cv_work.notify_one();
    return SPMV_OK;
}

spmv_status wait_ticket(spmv_server *S, int64_t ticket, double *latency) {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_error("spmv_server_wait: unknown ticket");
        return SPMV_ERR_INVALID_ARG;
    }
    Req *q = it->second;
    S->cv_done.wait(lk, [&] { return q->done; });
    if (latency) *latency = q->t_done - q->t_arr;
    const spmv_status st = q->st;
    if (st != SPMV_OK) set_error(q->msg);
    S->reqs.erase(it);
    delete q;
    return st;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

spmv_status spmv_server_create(const spmv_server_opts *opts, spmv_server_t *out) {
    if (!opts || !out || opts->budget_bytes <= 0 || opts->slots < 1 || opts->slots > 64 || opts->max_batch < 1 ||
        opts->max_batch > 1024) {
        set_error("spmv_server_create: budget > 0, 1 <= slots <= 64, 1 <= max_batch <= 1024");
        return SPMV_ERR_INVALID_ARG;
    }
    auto *S = new spmv_server();
    S->o = *opts;
    cudaGetDevice(&S->device);
    S->slots.resize(opts->slots);
    for (Slot &sl : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        sl.bs = batch_slot_new();
        if (e != cudaSuccess) {
            const spmv_status st = cuda_status(e, "spmv_server_create");
            spmv_server_destroy(S);
            return st;
        }
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return SPMV_OK;
}

spmv_status spmv_server_add(spmv_server_t S, spmv_handle h, int32_t *matrix_id) {
    if (!S || !h || !matrix_id) {
        set_error("spmv_server_add: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    if (!h->has_csr) {
        set_error("spmv_server_add: convert the matrix first");
        return SPMV_ERR_NOT_CONVERTED;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (!h->has_merge) SPMV_TRY(build_merge(h, MERGE_WARP_ITEMS, nullptr));
    SPMV_CUDA_TRY(cudaStreamSynchronize(nullptr));
    if (S->resident + h->bytes > S->o.budget_bytes) {
        set_error("spmv_server_add: the resident set would exceed the memory budget");
        return SPMV_ERR_OOM;
    }
    Mat M;
    M.h = h;
    M.bytes = h->bytes;
    S->mats.push_back(M);
    S->resident += h->bytes;
    S->st.resident_bytes = S->resident;
    *matrix_id = (int32_t)(S->mats.size() - 1);
    return SPMV_OK;
}

spmv_status spmv_server_submit(spmv_server_t S, const spmv_request *r, int64_t *ticket) {
    if (!S || !ticket) {
        set_error("spmv_server_submit: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    return submit_at(S, r, now_s(), ticket);
}

spmv_status spmv_server_wait(spmv_server_t S, int64_t ticket, double *latency_s) {
    if (!S) {
        set_error("spmv_server_wait: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    return wait_ticket(S, ticket, latency_s);
}

spmv_status spmv_server_replay(spmv_server_t S, int64_t n, const spmv_request *reqs, const double *arrival_s,
                               double *latency_s) {
    if (!S || n < 0 || (n > 0 && (!reqs || !arrival_s || !latency_s))) {
        set_error("spmv_server_replay: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    for (int64_t i = 1; i < n; ++i)
        if (arrival_s[i] < arrival_s[i - 1]) {
            set_error("spmv_server_replay: arrival times must be non-decreasing");
            return SPMV_ERR_INVALID_ARG;
        }
    std::vector<int64_t> tickets((size_t)n, 0);
    const double t0 = now_s() + 1e-3;
    spmv_status first = SPMV_OK;
    int64_t submitted = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double ta = t0 + arrival_s[i];
        while (now_s() < ta) {
        }
        const spmv_status st = submit_at(S, &reqs[i], ta, &tickets[i]);
        if (st != SPMV_OK) {
            first = st;
            break;
        }
        ++submitted;
    }
    for (int64_t i = 0; i < submitted; ++i) {
        const spmv_status st = wait_ticket(S, tickets[i], &latency_s[i]);
        if (st != SPMV_OK && first == SPMV_OK) first = st;
    }
    for (int64_t i = submitted; i < n; ++i) latency_s[i] = -1.0;
    return first;
}

spmv_status spmv_server_stats(spmv_server_t S, spmv_server_stats_t *out) {
    if (!S || !out) {
        set_error("spmv_server_stats: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    S->st.resident_bytes = S->resident;
    *out = S->st;
    return SPMV_OK;
}

spmv_status spmv_server_destroy(spmv_server_t S) {
    if (!S) return SPMV_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaError_t e = cudaSuccess;
    for (Slot &sl : S->slots) {
        if (sl.s) {
            const cudaError_t e2 = cudaStreamSynchronize(sl.s);
            if (e == cudaSuccess) e = e2;
        }
        batch_slot_free(sl.bs);
        if (sl.pin) cudaFreeHost(sl.pin);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    for (Mat &M : S->mats) dev_free(M.pr_x);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    if (e != cudaSuccess) return cuda_status(e, "spmv_server_destroy");
    return SPMV_OK;
}

}  // extern "C"
