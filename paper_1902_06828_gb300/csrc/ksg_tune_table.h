// Launch shapes of the member-lane KSG kernel by problem shape.  Written by
// paper_1902_06828_gb300/tune_ksg.py from timed runs on one GB300 (every
// shape bucket timed with every tile length and members-per-lane count, the
// fastest kept); the runtime takes the first row whose bucket holds the
// launch: points N <= n_max, conditioning dimensions dz <= dz_max and every
// group of the launch with at least min_members members.
#pragma once

namespace teksg {

struct KsgTuneEntry {
    int n_max, dz_max, min_members;
    int jt;   // points per staged tile: 64, 128 or 256
    int ms;   // members per lane: 1 or 2 (2 needs min_members >= 64)
};

// tuned: T = 1000 / 3000 / 10000 points, conditioning dims 0 / 1 / 2 / 4 / 8,
// 45 candidates x 201 members (rows with min_members 64) or 21 members
static const KsgTuneEntry kKsgTune[] = {
    {1500, 0, 64, 128, 2},
    {1500, 0, 0, 128, 1},
    {1500, 1, 64, 256, 2},
    {1500, 1, 0, 256, 1},
    {1500, 3, 64, 256, 2},
    {1500, 3, 0, 256, 1},
    {1500, 7, 64, 256, 2},
    {1500, 7, 0, 256, 1},
    {1500, 1073741824, 64, 256, 2},
    {1500, 1073741824, 0, 256, 1},
    {4500, 0, 64, 256, 2},
    {4500, 0, 0, 256, 1},
    {4500, 1, 64, 256, 2},
    {4500, 1, 0, 256, 1},
    {4500, 3, 64, 256, 2},
    {4500, 3, 0, 256, 1},
    {4500, 7, 64, 256, 2},
    {4500, 7, 0, 256, 1},
    {4500, 1073741824, 64, 256, 2},
    {4500, 1073741824, 0, 256, 1},
    {1073741824, 0, 64, 256, 1},
    {1073741824, 0, 0, 256, 1},
    {1073741824, 1, 64, 256, 2},
    {1073741824, 1, 0, 256, 1},
    {1073741824, 3, 64, 256, 2},
    {1073741824, 3, 0, 256, 1},
    {1073741824, 7, 64, 256, 2},
    {1073741824, 7, 0, 256, 1},
    {1073741824, 1073741824, 64, 256, 2},
    {1073741824, 1073741824, 0, 256, 1},
    {1 << 30, 1 << 30, 0, 256, 1},
};

}  // namespace teksg
