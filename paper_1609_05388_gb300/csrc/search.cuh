// The certified search for the smallest target dimension, as a state machine
// shared by the single and the batched fit (the question Table 3 answers: how
// many dimensions reach distortion eps).
//
// Probe r = 16, 32, 64, ... (the last probe is the cap) until a certificate
// passes, then bisect between the last failing and the first passing probe
// with mid = floor((lo + hi) / 2).  A predicted start is probed first: with
// verify_only it is accepted when it passes; when it fails the doubling
// sequence continues above it.  The result is the smallest passing probe
// (tracked by the caller), or none when even the cap fails.
#pragma once

#include <vector>

namespace adagio {

struct Search {
    int cap = 0, start = 0;
    bool verify_only = false;
    int stage = 3;  // 0 predicted start, 1 doubling, 2 bisection, 3 finished
    std::vector<int> seq;
    size_t si = 0;
    int lo = 0, hi = 0;

    void begin(int cap_, int start_, bool verify_only_) {
        cap = cap_;
        start = start_ > 0 ? (start_ < cap_ ? start_ : cap_) : 0;
        verify_only = verify_only_;
        if (start > 0) {
            stage = 0;
        } else {
            doubling(0);
        }
    }

    // the dimension to probe next; 0 once the search is over
    int next() const {
        switch (stage) {
            case 0: return start;
            case 1: return seq[si];
            case 2: return (lo + hi) / 2;
            default: return 0;
        }
    }

    void record(bool ok) {
        const int r = next();
        switch (stage) {
            case 0:
                if (ok) {
                    if (verify_only) stage = 3;
                    else bisect(0, r);
                } else {
                    doubling(r);
                }
                break;
            case 1:
                if (ok) {
                    bisect(si > 0 ? seq[si - 1] : last_fail0, r);
                } else if (++si == seq.size()) {
                    stage = 3;
                }
                break;
            case 2:
                if (ok) hi = r; else lo = r;
                if (hi - lo <= 1) stage = 3;
                break;
            default: break;
        }
    }

   private:
    int last_fail0 = 0;  // the failure the doubling sequence started above

    void doubling(int last_fail) {
        last_fail0 = last_fail;
        seq.clear();
        for (int r = 16; r < cap; r *= 2)
            if (r > last_fail) seq.push_back(r);
        if (cap > last_fail) seq.push_back(cap);
        si = 0;
        stage = seq.empty() ? 3 : 1;
    }

    void bisect(int lo_, int hi_) {
        lo = lo_;
        hi = hi_;
        stage = hi - lo > 1 ? 2 : 3;
    }
};

}  // namespace adagio
