// gl_profile.cuh -- launch accounting and CUDA-event timing of one named kernel
// class (instrumentation for measurement; not part of the method).
//
// Direct launches take an event pair from a pool and are summed at the next
// harvest.  Launches captured into a CUDA graph keep their event pair for the
// life of the graph; the graph's owner harvests those pairs after every replay.
// gl_profile_begin/end bump `generation` whenever graphs may hold event nodes
// of the old event pool or must gain some, so those graphs are captured again;
// counting launches only (no class) leaves graphs without event nodes alone.
#pragma once

#include <atomic>
#include <string>
#include <vector>

#include "gl_common.cuh"

namespace gl {

struct Profiler {
    std::atomic<int64_t> launches{0};  // hot-path kernel launches since gl_profile_begin
    int64_t generation = 0;
    // timed class under which the graphs of the current generation are captured
    // ("" = none: such graphs hold no event nodes and survive a change to "" )
    std::string graph_state;
    // a new generation unless both the graphs' state and the new one time nothing
    void retarget(const std::string &state) {
        if (!(graph_state.empty() && state.empty())) generation += 1;
        graph_state = state;
    }
    bool active = false;
    std::string name;                  // kernel class timed with events ("" = none)
    std::vector<cudaEvent_t> ev;       // 2 per slot
    std::vector<double> slot_bytes, slot_flops;
    std::vector<int> free_slots, pending;
    std::vector<int> *capture = nullptr;  // slots of the graph being captured
    double total_ms = 0, total_bytes = 0, total_flops = 0;
    double last_flops = 0;  // total_flops of the last ended profile
    int64_t timed = 0, dropped = 0;

    bool timing(const char *cls) const { return active && !name.empty() && name == cls; }
    // sums the elapsed time of the given slots (their events have completed)
    void harvest(const std::vector<int> &slots) {
        for (int sl : slots) {
            float t = 0;
            if (cudaEventElapsedTime(&t, ev[2 * sl], ev[2 * sl + 1]) == cudaSuccess) {
                total_ms += t;
                total_bytes += slot_bytes[sl];
                total_flops += slot_flops[sl];
                ++timed;
            }
        }
    }
    void harvest_direct() {
        harvest(pending);
        free_slots.insert(free_slots.end(), pending.begin(), pending.end());
        pending.clear();
    }
};
Profiler &profiler();

inline void note_launch(int k = 1) { profiler().launches.fetch_add(k, std::memory_order_relaxed); }

// Brackets one launch: records events around it when its class is being timed.
// alg_flops: the launch's arithmetic (flops, an FMA counted as 2) where a kernel
// may be bound by an arithmetic pipe rather than by memory; 0 where not counted.
class ProfScope {
   public:
    ProfScope(const char *cls, double alg_bytes, cudaStream_t s, double alg_flops = 0) : s_(s) {
        Profiler &p = profiler();
        note_launch();
        if (!p.timing(cls)) return;
        if (p.free_slots.empty()) {
            ++p.dropped;
            return;
        }
        slot_ = p.free_slots.back();
        p.free_slots.pop_back();
        p.slot_bytes[slot_] = alg_bytes;
        p.slot_flops[slot_] = alg_flops;
        graph_ = p.capture != nullptr;
        if (graph_)
            p.capture->push_back(slot_);
        else
            p.pending.push_back(slot_);
        record(p.ev[2 * slot_]);
    }
    ~ProfScope() {
        if (slot_ >= 0) record(profiler().ev[2 * slot_ + 1]);
    }

   private:
    // inside stream capture an event record becomes a timing node of the graph
    // only with cudaEventRecordExternal
    void record(cudaEvent_t e) {
        if (graph_)
            cudaEventRecordWithFlags(e, s_, cudaEventRecordExternal);
        else
            cudaEventRecord(e, s_);
    }

    cudaStream_t s_;
    int slot_ = -1;
    bool graph_ = false;
};

}  // namespace gl
