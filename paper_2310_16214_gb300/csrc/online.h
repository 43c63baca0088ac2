// Online tuning across calls (online.cu).
#pragma once

#include "internal.h"

namespace bplg {

// What a call must do for the online tuner: applies = the plan came from it;
// e0/e1 set = record e0 before the launch and pass the launch's status to
// online_launched (which records e1).
struct OnlineTicket {
    bool applies = false;
    void *state = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

int online_set(bool enable, int budget, uint64_t seed);
int online_plan(int op, int dtype, int64_t n, int64_t batch, bplg_plan *out, OnlineTicket *t);
void online_launched(const OnlineTicket &t, cudaStream_t s, int launch_rc);
int online_status(int op, int dtype, int64_t n, int64_t batch, int32_t *evaluations, int32_t *finished,
                  bplg_plan *best);

}  // namespace bplg
