// Served execution: continuous batching of binarization requests.
//
// Requests (device-resident images) are queued by bz_server_submit.  A
// scheduler thread admits queued requests in FIFO order while the summed
// image+output bytes of the requests on the device stay within the HBM
// budget and fewer than max_slots requests are in flight, groups the
// admitted requests of one precision into a batch and launches it through an
// idle batch slot on that slot's own stream (the batched persistent kernels
// of batch.cu).  Several batches are in flight at once on different streams,
// so requests that arrive while others run are admitted as soon as budget and
// a slot free up, and their work overlaps on the device.  The scheduler
// holds the server lock only to pick requests and to retire finished
// batches; batches are built and launched outside it.  Each launch ends with
// a host callback on its stream that wakes the scheduler (the callback only
// sets a flag and signals), and completion is confirmed with the lane's CUDA
// event; bz_server_wait blocks on a condition variable.
//
// In-place requests (out == image, out_pitch == in_pitch; Sauvola and
// Niblack) hold the image plus the scratch of binarize_inplace: row bands
// when image + row scratch fits the budget at admission, else column bands
// (binarize_inplace_cols, the exchanged axes of Sec. 3.3) when their smaller
// scratch fits; a request that fits neither waits at the head of the queue.
// They run on the lane's stream after the lane's batch.
//
// Host-side fault injection for tests (environment variable BZ_FAULT):
//   "launch"     every batch launch reports BZ_ECUDA without touching the GPU
//   "slow:<ms>"  completions are reported <ms> milliseconds late
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_internal.h"

namespace bz {

enum ReqState { RS_QUEUED, RS_RUNNING, RS_DONE };

enum Orient { OR_NONE, OR_ROWS, OR_COLS };  // in-place orientation (OR_NONE: separate output)

struct Request {
    bz_job job;
    bz_precision prec;
    int64_t bytes;       // bytes held on the device while running
    ReqState state;
    bz_status result;
    bool cancelled;
    bool inplace;
    int64_t bytes_rows, bytes_cols;  // in-place: image + scratch of each orientation (-1: not offered)
};

struct ExecLane {
    BatchSlot slot;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;      // a batch was handed to this lane
    bool launched = false;  // ... and launched (event recorded, callback queued)
    bool failed = false;
    bool signalled = false;  // the stream's callback ran
    std::vector<uint64_t> tickets;
    std::vector<bz_job> jobs;      // separate-output jobs: one batch
    std::vector<bz_job> ip_jobs;   // in-place jobs, run one by one after it
    std::vector<int> ip_orient;
    bz_precision prec = BZ_FP64;
    std::chrono::steady_clock::time_point ready_at;
    bz_server *srv = nullptr;
};

}  // namespace bz

struct bz_server {
    int64_t budget = 0;
    int32_t max_slots = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::condition_variable cv_work;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, bz::Request> reqs;
    uint64_t next_ticket = 1;
    int64_t inflight_bytes = 0;
    int32_t inflight = 0;
    std::vector<bz::ExecLane *> lanes;
    std::thread sched;
    bool stop = false;
    bool fault_launch = false;
    int fault_slow_ms = 0;
};

namespace bz {

static int64_t job_bytes(const bz_job &j)
{
    return j.H * j.in_pitch + j.H * j.out_pitch;
}

static bool is_inplace(const bz_job &j)
{
    return j.out == j.image && j.out_pitch == j.in_pitch;
}

static bz_status run_inplace(const bz_job &j, int orient, bz_precision prec, cudaStream_t s)
{
    const int32_t m = j.method == BZ_SAUVOLA ? 0 : 1;
    if (orient == OR_ROWS)
        return binarize_inplace(m, j.out, j.H, j.W, j.in_pitch, j.h, j.w, j.k, j.R, 0, prec, s);
    return binarize_inplace_cols(m, j.out, j.H, j.W, j.in_pitch, j.h, j.w, j.k, j.R, 0, prec, s);
}

// Completes the lanes whose batch finished; called with srv->mu held.
static void reap(bz_server *srv)
{
    const auto now = std::chrono::steady_clock::now();
    for (ExecLane *L : srv->lanes) {
        if (!L->busy || (!L->launched && !L->failed))
            continue;
        bz_status result = BZ_OK;
        if (!L->failed) {
            const cudaError_t q = cudaEventQuery(L->ev);  // never blocks
            if (q == cudaErrorNotReady)
                continue;
            if (q != cudaSuccess)
                result = BZ_ECUDA;
        } else {
            result = BZ_ECUDA;
        }
        if (srv->fault_slow_ms > 0) {
            if (L->ready_at.time_since_epoch().count() == 0)
                L->ready_at = now + std::chrono::milliseconds(srv->fault_slow_ms);
            if (now < L->ready_at)
                continue;
        }
        for (uint64_t t : L->tickets) {
            auto it = srv->reqs.find(t);
            if (it == srv->reqs.end())
                continue;
            it->second.state = RS_DONE;
            it->second.result = it->second.cancelled ? BZ_ECANCELLED : result;
            srv->inflight_bytes -= it->second.bytes;
            srv->inflight -= 1;
        }
        L->tickets.clear();
        L->jobs.clear();
        L->ip_jobs.clear();
        L->ip_orient.clear();
        L->busy = false;
        L->launched = false;
        L->failed = false;
        L->signalled = false;
        L->ready_at = {};
    }
}

// Hands queued requests to idle lanes (FIFO under the budget and the slot
// cap); called with srv->mu held.  Returns the lanes to launch.
static std::vector<ExecLane *> pick(bz_server *srv)
{
    std::vector<ExecLane *> ready;
    for (ExecLane *L : srv->lanes) {
        if (L->busy)
            continue;
        if (srv->queue.empty())
            break;
        bz_precision prec = BZ_FP64;
        bool have_prec = false;
        // requests of another precision wait for a later batch
        for (auto it = srv->queue.begin(); it != srv->queue.end();) {
            Request &r = srv->reqs[*it];
            if (have_prec && r.prec != prec) {
                ++it;
                continue;
            }
            if (srv->inflight >= srv->max_slots)
                break;
            const int64_t room = srv->budget - srv->inflight_bytes;
            int orient = OR_NONE;
            if (r.inplace) {
                if (r.bytes_rows >= 0 && r.bytes_rows <= room)
                    orient = OR_ROWS;  // faster: whole-width launches
                else if (r.bytes_cols >= 0 && r.bytes_cols <= room)
                    orient = OR_COLS;  // less scratch
                else
                    break;  // head-of-line: keep FIFO order under the budget
                r.bytes = orient == OR_ROWS ? r.bytes_rows : r.bytes_cols;
            } else if (r.bytes > room) {
                break;
            }
            prec = r.prec;
            have_prec = true;
            r.state = RS_RUNNING;
            srv->inflight_bytes += r.bytes;
            srv->inflight += 1;
            if (r.inplace) {
                L->ip_jobs.push_back(r.job);
                L->ip_orient.push_back(orient);
            } else {
                L->jobs.push_back(r.job);
            }
            L->tickets.push_back(*it);
            it = srv->queue.erase(it);
        }
        if (L->tickets.empty())
            break;
        L->prec = prec;
        L->busy = true;
        L->launched = false;
        L->failed = false;
        L->signalled = false;
        ready.push_back(L);
    }
    return ready;
}

// Host callback at the end of a lane's batch: wake the scheduler (no CUDA
// call here).
static void CUDART_CB lane_done(void *arg)
{
    ExecLane *L = static_cast<ExecLane *>(arg);
    std::lock_guard<std::mutex> lk(L->srv->mu);
    L->signalled = true;
    L->srv->cv_work.notify_one();
}

static void scheduler(bz_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        reap(srv);
        std::vector<ExecLane *> ready = pick(srv);
        srv->cv_done.notify_all();
        if (!ready.empty()) {
            // build and launch outside the lock: submitters and waiters
            // proceed meanwhile (a lane's fields belong to the scheduler
            // while it is busy and not yet launched)
            lk.unlock();
            for (ExecLane *L : ready) {
                bool ok = !srv->fault_launch;
                if (ok && !L->jobs.empty())
                    ok = run_batch(L->slot, L->jobs.data(), (int32_t)L->jobs.size(), L->prec, L->stream) ==
                         BZ_OK;
                for (size_t q = 0; ok && q < L->ip_jobs.size(); q++)
                    ok = run_inplace(L->ip_jobs[q], L->ip_orient[q], L->prec, L->stream) == BZ_OK;
                if (ok)
                    ok = cudaEventRecord(L->ev, L->stream) == cudaSuccess &&
                         cudaLaunchHostFunc(L->stream, lane_done, L) == cudaSuccess;
                lk.lock();
                if (ok)
                    L->launched = true;
                else
                    L->failed = true;
                lk.unlock();
            }
            lk.lock();
            continue;  // reap failed launches and pick again
        }
        bool any_busy = false;
        for (ExecLane *L : srv->lanes)
            any_busy |= L->busy;
        if (srv->stop && srv->queue.empty() && !any_busy)
            break;
        // woken by a submission, a completion callback (which sets its flag
        // and signals under the lock, so no wake-up is lost) or shutdown; the
        // timeout paces BZ_FAULT=slow and bounds anything unforeseen
        srv->cv_work.wait_for(lk, std::chrono::milliseconds(srv->fault_slow_ms > 0 ? 1 : 50));
    }
    srv->cv_done.notify_all();
}

}  // namespace bz

using namespace bz;

extern "C" {

bz_status bz_server_create(int64_t hbm_budget_bytes, int32_t max_slots, bz_server **out)
{
    if (!out || hbm_budget_bytes <= 0 || max_slots < 1)
        return BZ_EINVAL;
    *out = nullptr;
    bz_server *srv = new (std::nothrow) bz_server();
    if (!srv)
        return BZ_ENOMEM;
    srv->budget = hbm_budget_bytes;
    srv->max_slots = max_slots;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return BZ_ECUDA;
    }
    const char *f = getenv("BZ_FAULT");
    if (f) {
        if (strcmp(f, "launch") == 0)
            srv->fault_launch = true;
        else if (strncmp(f, "slow:", 5) == 0)
            srv->fault_slow_ms = atoi(f + 5);
    }
    const int nlanes = 4;  // batches in flight at once (independent streams)
    for (int i = 0; i < nlanes; i++) {
        ExecLane *L = new ExecLane();
        L->srv = srv;
        if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming) != cudaSuccess) {
            delete L;
            bz_server_destroy(srv);
            return BZ_ECUDA;
        }
        srv->lanes.push_back(L);
    }
    srv->sched = std::thread(scheduler, srv);
    *out = srv;
    return BZ_OK;
}

bz_status bz_server_submit(bz_server *srv, const bz_job *job, bz_precision precision,
                           uint64_t *ticket)
{
    if (!srv || !job || !ticket)
        return BZ_EINVAL;
    if (precision != BZ_FP64 && precision != BZ_FP32 && precision != BZ_FP64_DIRECT)
        return BZ_EINVAL;
    Request r{*job, precision, 0, RS_QUEUED, BZ_OK, false, is_inplace(*job), -1, -1};
    if (r.inplace) {
        const bz_job &j = *job;
        bz_status st = check_image(j.image, j.H, j.W, j.in_pitch, j.h, j.w);
        if (st != BZ_OK)
            return st;
        if ((j.method != BZ_SAUVOLA && j.method != BZ_NIBLACK) ||
            !finite_params(j.method == BZ_SAUVOLA ? 0 : 1, j.k, j.R))
            return BZ_EINVAL;
        const int64_t img = j.H * j.in_pitch;
        const int64_t sr = bz_inplace_scratch_bytes(j.H, j.W, j.h, 0);
        const int64_t sc = bz_inplace_cols_scratch_bytes(j.H, j.W, j.w, 0);
        r.bytes_rows = sr < 0 ? -1 : img + sr;
        r.bytes_cols = sc < 0 ? -1 : img + sc;
        const int64_t least = r.bytes_cols >= 0 && r.bytes_cols < r.bytes_rows ? r.bytes_cols : r.bytes_rows;
        if (least < 0)
            return BZ_EINVAL;
        if (least > srv->budget)
            return BZ_EBUDGET;
        r.bytes = least;
    } else {
        const bz_status st = validate_job(*job);
        if (st != BZ_OK)
            return st;
        r.bytes = job_bytes(*job);
        if (r.bytes > srv->budget)
            return BZ_EBUDGET;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop)
        return BZ_EINVAL;
    const uint64_t t = srv->next_ticket++;
    srv->reqs[t] = r;
    srv->queue.push_back(t);
    *ticket = t;
    srv->cv_work.notify_one();
    return BZ_OK;
}

bz_status bz_server_cancel(bz_server *srv, uint64_t ticket)
{
    if (!srv)
        return BZ_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end())
        return BZ_EINVAL;
    if (it->second.state == RS_QUEUED) {
        for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
            if (*q == ticket) {
                srv->queue.erase(q);
                break;
            }
        it->second.state = RS_DONE;
        it->second.result = BZ_ECANCELLED;
        srv->cv_done.notify_all();
        return BZ_OK;
    }
    // in flight: the GPU work cannot be recalled; it completes and the
    // request reports BZ_ECANCELLED
    if (it->second.state == RS_RUNNING) {
        it->second.cancelled = true;
        return BZ_OK;
    }
    return BZ_EINVAL;  // already finished
}

bz_status bz_server_wait(bz_server *srv, uint64_t ticket, int32_t timeout_ms)
{
    if (!srv)
        return BZ_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end())
        return BZ_EINVAL;
    auto done = [&] { return srv->reqs[ticket].state == RS_DONE; };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, done);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        Request &r = srv->reqs[ticket];
        if (r.state == RS_QUEUED) {
            // never started: dropped, its buffers are free now
            for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
                if (*q == ticket) {
                    srv->queue.erase(q);
                    break;
                }
            srv->reqs.erase(ticket);
            return BZ_ETIMEOUT;
        }
        // running: the GPU work cannot be recalled.  The request is
        // cancelled and keeps its ticket: its buffers stay in use until a
        // later wait on the ticket returns BZ_ECANCELLED (or the server is
        // destroyed)
        r.cancelled = true;
        return BZ_ETIMEOUT;
    }
    const bz_status result = srv->reqs[ticket].result;
    srv->reqs.erase(ticket);
    return result;
}

bz_status bz_server_destroy(bz_server *srv)
{
    if (!srv)
        return BZ_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (uint64_t t : srv->queue) {
            srv->reqs[t].state = RS_DONE;
            srv->reqs[t].result = BZ_ECANCELLED;
        }
        srv->queue.clear();
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    if (srv->sched.joinable())
        srv->sched.join();
    for (ExecLane *L : srv->lanes) {
        if (L->stream)
            cudaStreamSynchronize(L->stream);
        if (L->ev)
            cudaEventDestroy(L->ev);
        if (L->stream)
            cudaStreamDestroy(L->stream);
        delete L;
    }
    delete srv;
    return BZ_OK;
}

}  // extern "C"
