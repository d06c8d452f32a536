// Request scheduling of the serving path, free of CUDA: the state machine that the server's
// scheduler thread runs (serve.cu) and that a CPU test drives through a fake device.
//
// A request moves QUEUED -> (admitted) RUNNING -> COPYING -> DONE -> RELEASED:
//   admission  in arrival order under a device-memory budget; a hard request also takes a slot of
//              the persistent kernel's request table (soft requests run as their own kernels and
//              take none). The first queued request that does not fit the budget, finds no slot
//              or whose device allocation fails stops admission until a later pass: requests never
//              overtake one another, so a large request cannot be starved by small ones. A
//              cancelled request (still QUEUED) is dropped from the queue.
//   running    the device evaluates its work units; when they are all done the scheduler queues
//              the copies of the results (COPYING), and when those have landed the request is
//              DONE: its memory and slot return to the budget and the free list.
//   relaunch   the persistent kernel leaves after an idle limit; a pass that finds units waiting
//              and no kernel live launches it again.
// A device error while copying marks the request and makes the scheduler fatal (later
// submissions are refused by the server).
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <memory>
#include <vector>

namespace rs {
namespace sched {

enum : int { QUEUED = 0, RUNNING = 2, COPYING = 3, DONE = 4, RELEASED = 5 };

// The part of a request the scheduler decides on; the server's request type derives from it.
struct Core {
    uint64_t ticket = 0;
    size_t device_bytes = 0;
    bool needs_slot = true;      // hard requests: a slot of the persistent kernel's request table
    int slot = -1;
    int state = QUEUED;
    int status = 0;              // 0 or an rs_status error
};

// B, the device side:
//   bool admit(R &r)        allocate r's device memory, upload and prepare it (r.slot is set when it
//                           needs one) and set r.state to RUNNING (work published) or COPYING (no
//                           work: the results are already being copied); false if the allocation
//                           failed (nothing taken: tried again on a later pass)
//   bool kernel_live()      the persistent kernel is running (may notice that it has exited)
//   void launch_kernel()
//   bool units_done(R &r)   every work unit of a RUNNING request has finished
//   void start_copy_out(R &r)
//   int  copies_done(R &r)  1 landed, 0 not yet, < 0 a device error (an rs_status)
//   void release(R &r)      free r's device memory
template <class R, class B>
struct Scheduler {
    size_t budget = 0, used = 0;
    std::vector<int> free_slots;
    std::deque<std::shared_ptr<R>> queued;
    std::vector<std::shared_ptr<R>> active;
    int fatal = 0;
    int64_t launches = 0;

    void init(size_t budget_bytes, int slots)
    {
        budget = budget_bytes;
        free_slots.clear();
        for (int i = slots - 1; i >= 0; --i) free_slots.push_back(i);
    }

    bool idle() const { return queued.empty() && active.empty(); }

    // Cancel a request that has not been admitted. False if it already was.
    bool cancel(R &r, int cancelled_status)
    {
        if (r.state != QUEUED) return false;
        r.status = cancelled_status;
        r.state = DONE;
        return true;
    }

    // One pass of the scheduler; returns whether anything changed.
    bool step(B &b)
    {
        bool progress = false;
        while (!queued.empty()) {                 // admission, arrival order
            std::shared_ptr<R> r = queued.front();
            if (r->state >= DONE) {               // cancelled while queued
                queued.pop_front();
                continue;
            }
            if (used + r->device_bytes > budget || (r->needs_slot && free_slots.empty())) break;
            if (r->needs_slot) r->slot = free_slots.back();
            if (!b.admit(*r)) {                   // allocation failed: retried on a later pass
                r->slot = -1;
                break;
            }
            if (r->needs_slot) free_slots.pop_back();
            used += r->device_bytes;
            queued.pop_front();
            active.push_back(r);
            progress = true;
        }
        bool waiting = false;                     // units published and not all done
        for (auto &r : active) waiting |= r->state == RUNNING;
        if (waiting && !b.kernel_live()) {
            b.launch_kernel();
            ++launches;
            progress = true;
        }
        for (auto &r : active) {                  // completions
            if (r->state == RUNNING && b.units_done(*r)) {
                b.start_copy_out(*r);
                r->state = COPYING;
                progress = true;
            }
            if (r->state == COPYING) {
                const int q = b.copies_done(*r);
                if (q > 0) {
                    b.release(*r);
                    used -= r->device_bytes;
                    if (r->slot >= 0) free_slots.push_back(r->slot);
                    r->state = DONE;
                    progress = true;
                } else if (q < 0) {
                    fatal = q;
                    r->status = q;
                    r->state = DONE;
                    progress = true;
                }
            }
        }
        active.erase(std::remove_if(active.begin(), active.end(),
                                    [](const std::shared_ptr<R> &r) { return r->state >= DONE; }),
                     active.end());
        return progress;
    }
};

}  // namespace sched
}  // namespace rs
