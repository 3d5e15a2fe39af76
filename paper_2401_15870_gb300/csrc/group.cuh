// group.cuh -- asynchronous form of the group update, for the request loop
// (server.cu).
#pragma once
#include "dfpr.h"

// launch an update of the members (indices into the group; NULL: every graph)
// on the group's stream and return without waiting; one at a time per group
pr_status group_launch(pr_group* q, pr_method method, double alpha, double tau, const pr_options* opts,
                       const int32_t* members, int32_t nm);
// the launched update has finished (never blocks)
bool group_done(pr_group* q);
// wait for it and write the members' stats (indexed by group position)
pr_status group_complete(pr_group* q, pr_stats* stats);
