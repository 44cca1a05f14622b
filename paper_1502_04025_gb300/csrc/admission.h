// Admission policy of the serving loop (host only; no CUDA, so that the
// rules are testable on their own).
//
// A batch is a lead request plus every queued request that may share its
// solve (same gauge field and parameters), up to max_rhs right-hand sides.
// prepare(lead, total_rhs) makes every allocation the batch's solve needs and
// returns QDD_OK, QDD_EBUDGET when the budget refuses it, or another error.
// The lead is the head of the queue; while the head does not fit, later
// requests that fit may go first, at most max_bypass of them per head, after
// which admission waits for the head.  A batch that does not fit is retried
// with its lead alone.  With nothing running, a head that does not fit can
// never fit and is rejected; a lead whose preparation fails otherwise is
// rejected with that status.
#pragma once

#include <algorithm>
#include <deque>
#include <memory>
#include <vector>

#include "qdd.h"

namespace qdd {

enum class Admit { kBatch, kWait, kReject };

template <typename Req>
struct AdmitResult {
    Admit what = Admit::kWait;
    std::vector<std::shared_ptr<Req>> batch;  // kBatch: the requests to solve together (lead first)
    std::shared_ptr<Req> rejected;            // kReject: the request to fail
    qdd_status status = QDD_OK;               // kReject: its status
};

// Req needs an int member `bypassed`; nrhs_of(r), same(a, b) and
// prepare(lead, total) are callables.
template <typename Req, typename NrhsFn, typename SameFn, typename PrepareFn>
AdmitResult<Req> admit(std::deque<std::shared_ptr<Req>> &queue, bool any_running, int max_rhs, int max_bypass,
                       NrhsFn nrhs_of, SameFn same, PrepareFn prepare)
{
    AdmitResult<Req> res;
    if (queue.empty()) return res;
    auto head = queue.front();
    const size_t nlead = head->bypassed < max_bypass ? queue.size() : 1;
    qdd_status ps = QDD_EBUDGET;
    std::vector<std::shared_ptr<Req>> cand;
    std::shared_ptr<Req> lead;
    for (size_t li = 0; li < nlead && ps == QDD_EBUDGET; li++) {
        lead = queue[li];
        cand.assign(1, lead);
        int total = nrhs_of(*lead);
        for (auto &r : queue)
            if (r != lead && same(*r, *lead) && total + nrhs_of(*r) <= max_rhs) {
                cand.push_back(r);
                total += nrhs_of(*r);
            }
        ps = prepare(*lead, total);
        if (ps == QDD_EBUDGET && cand.size() > 1) {
            cand.resize(1);
            ps = prepare(*lead, nrhs_of(*lead));
        }
    }
    if (ps == QDD_OK) {
        if (std::find(cand.begin(), cand.end(), head) == cand.end()) head->bypassed++;
        for (auto &r : cand) queue.erase(std::find(queue.begin(), queue.end(), r));
        res.what = Admit::kBatch;
        res.batch = std::move(cand);
        return res;
    }
    if (ps != QDD_EBUDGET || !any_running) {
        res.what = Admit::kReject;
        res.rejected = ps != QDD_EBUDGET ? lead : head;
        res.status = ps;
        queue.erase(std::find(queue.begin(), queue.end(), res.rejected));
        return res;
    }
    return res;  // kWait
}

}  // namespace qdd
