// A fake device for the serving scheduler (test infrastructure): the scheduler of the library
// (serve_sched.h, the same header serve.cu runs) driven on the CPU. Device memory allocations
// succeed or fail as scripted, the persistent "kernel" completes work units between scheduler
// passes in the device's claim order (the request with the fewest unclaimed units first, the
// oldest among equals), result copies land one pass after they start, and a chosen request's
// copies can report a device error. A C interface for ctypes.
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "serve_sched.h"

namespace {

using namespace rs::sched;

struct FReq : Core {
    int units = 0, done_units = 0, copy_wait = 0;
};

struct Fake {
    std::deque<int> alloc_script;         // 1 succeed, 0 fail; empty: succeed
    bool kernel = false;
    int idle_ticks = 0;
    uint64_t fail_copy = 0;               // ticket whose copies report a device error
    std::vector<uint64_t> admitted, released;
    std::vector<FReq *> running;          // published work, in admission order

    bool admit(FReq &r)
    {
        int ok = 1;
        if (!alloc_script.empty()) {
            ok = alloc_script.front();
            alloc_script.pop_front();
        }
        if (!ok) return false;
        admitted.push_back(r.ticket);
        if (r.units > 0) {
            r.state = RUNNING;
            running.push_back(&r);
        } else {
            r.state = COPYING;
            r.copy_wait = 1;
        }
        return true;
    }
    bool kernel_live() { return kernel; }
    void launch_kernel() { kernel = true; idle_ticks = 0; }
    bool units_done(FReq &r) { return r.done_units >= r.units; }
    void start_copy_out(FReq &r)
    {
        r.copy_wait = 1;
        for (size_t i = 0; i < running.size(); ++i)
            if (running[i] == &r) { running.erase(running.begin() + i); break; }
    }
    int copies_done(FReq &r)
    {
        if (r.ticket == fail_copy) return -5;
        if (r.copy_wait > 0) { --r.copy_wait; return 0; }
        return 1;
    }
    void release(FReq &r) { released.push_back(r.ticket); }

    // The device between two scheduler passes: `n` units claimed one at a time, each from the
    // running request with the fewest unclaimed units (oldest among equals). The kernel leaves
    // after two ticks with nothing to claim.
    void tick(int n)
    {
        if (!kernel) return;
        bool any = false;
        for (int k = 0; k < n; ++k) {
            FReq *best = nullptr;
            for (FReq *r : running) {
                const int left = r->units - r->done_units;
                if (left > 0 && (!best || left < best->units - best->done_units)) best = r;
            }
            if (!best) break;
            ++best->done_units;
            any = true;
        }
        if (any) idle_ticks = 0;
        else if (++idle_ticks >= 2) kernel = false;
    }
};

struct Sim {
    Scheduler<FReq, Fake> sch;
    Fake dev;
    std::map<uint64_t, std::shared_ptr<FReq>> all;
    uint64_t next = 1;
};

}  // namespace

extern "C" {

void *fs_create(uint64_t budget, int slots)
{
    auto *s = new Sim();
    s->sch.init(budget, slots);
    return s;
}
void fs_destroy(void *h) { delete static_cast<Sim *>(h); }

uint64_t fs_submit(void *h, uint64_t bytes, int units, int needs_slot)
{
    auto *s = static_cast<Sim *>(h);
    auto r = std::make_shared<FReq>();
    r->ticket = s->next++;
    r->device_bytes = bytes;
    r->units = units;
    r->needs_slot = needs_slot != 0;
    s->all[r->ticket] = r;
    s->sch.queued.push_back(r);
    return r->ticket;
}

int fs_cancel(void *h, uint64_t t)
{
    auto *s = static_cast<Sim *>(h);
    return s->sch.cancel(*s->all.at(t), -8) ? 1 : 0;
}

void fs_script_alloc(void *h, int ok) { static_cast<Sim *>(h)->dev.alloc_script.push_back(ok); }
void fs_fail_copy(void *h, uint64_t t) { static_cast<Sim *>(h)->dev.fail_copy = t; }
int fs_step(void *h) { auto *s = static_cast<Sim *>(h); return s->sch.step(s->dev) ? 1 : 0; }
void fs_device_tick(void *h, int units) { static_cast<Sim *>(h)->dev.tick(units); }

int fs_state(void *h, uint64_t t) { return static_cast<Sim *>(h)->all.at(t)->state; }
int fs_status(void *h, uint64_t t) { return static_cast<Sim *>(h)->all.at(t)->status; }
int fs_slot(void *h, uint64_t t) { return static_cast<Sim *>(h)->all.at(t)->slot; }
uint64_t fs_used(void *h) { return static_cast<Sim *>(h)->sch.used; }
int fs_free_slots(void *h) { return (int)static_cast<Sim *>(h)->sch.free_slots.size(); }
int64_t fs_launches(void *h) { return static_cast<Sim *>(h)->sch.launches; }
int fs_fatal(void *h) { return static_cast<Sim *>(h)->sch.fatal; }
int fs_kernel_live(void *h) { return static_cast<Sim *>(h)->dev.kernel ? 1 : 0; }
int fs_idle(void *h) { return static_cast<Sim *>(h)->sch.idle() ? 1 : 0; }

int fs_admitted(void *h, uint64_t *out, int cap)
{
    auto &v = static_cast<Sim *>(h)->dev.admitted;
    for (int i = 0; i < (int)v.size() && i < cap; ++i) out[i] = v[i];
    return (int)v.size();
}
int fs_released(void *h, uint64_t *out, int cap)
{
    auto &v = static_cast<Sim *>(h)->dev.released;
    for (int i = 0; i < (int)v.size() && i < cap; ++i) out[i] = v[i];
    return (int)v.size();
}

}  // extern "C"
