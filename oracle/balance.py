"""Balancer oracle (TEST INFRASTRUCTURE ONLY): plain-Python restatements of
the two Charm++ strategies the paper uses (Sec. VI) and of the initial
block placement.

Costs are FP64 (Python floats); every load is accumulated in the order stated
below, so an implementation that performs the same FP64 additions in the same
order reproduces these assignments bit for bit.

  static_blocks  -- initial placement: processor p owns a contiguous run of
                    VPs, as the sub-domains 0000 1111 2222 3333 of Table V.
  greedy         -- GreedyLB (Sec. VI-A): "always assigns the heaviest
                    object to the least loaded processor", ignoring where the
                    objects currently are.
  refine_swap    -- RefineSwapLB (Sec. VI-B): moves objects off the most
                    overloaded processor toward the average, and swaps
                    objects when no single move fits.
  greedy_ordered -- GreedyLB's rule (each object to the least loaded
                    processor) with the objects taken in a given order
                    instead of heaviest first: Graham's list scheduling.
"""
import heapq


def static_blocks(nvps, nbins):
    """VP v goes to bin floor(v * nbins / nvps): contiguous, sizes differ by <= 1."""
    return [(v * nbins) // nvps for v in range(nvps)]


def bin_loads(costs, assign, nbins):
    """Per-bin FP64 sum, VPs added in increasing id order."""
    loads = [0.0] * nbins
    for v, b in enumerate(assign):
        loads[b] += costs[v]
    return loads


def total_load(loads):
    """Sum of the per-bin loads, bins in increasing id order: the numerator
    of the mean load per processor that RefineSwapLB balances toward
    (Sec. VI-B).  Equal to the sum of all costs up to rounding."""
    total = 0.0
    for x in loads:
        total += x
    return total


def max_over_mean(costs, assign, nbins):
    loads = bin_loads(costs, assign, nbins)
    mean = total_load(loads) / nbins
    return max(loads) / mean if mean > 0 else 1.0


def migrations(old, new):
    return sum(1 for a, b in zip(old, new) if a != b)


def greedy(costs, nbins):
    """GreedyLB.  Order VPs by (cost descending, id ascending); give each in
    turn to the bin with the least load so far (ties: lowest bin id); a bin's
    load is the FP64 sum of its VPs' costs in assignment order."""
    order = sorted(range(len(costs)), key=lambda v: (-costs[v], v))
    heap = [(0.0, b) for b in range(nbins)]
    heapq.heapify(heap)
    assign = [0] * len(costs)
    for v in order:
        load, b = heapq.heappop(heap)
        assign[v] = b
        heapq.heappush(heap, (load + costs[v], b))
    return assign


def greedy_ordered(costs, nbins, order):
    """Objects in the given order (a permutation of VP ids), each to the bin
    with the least load so far (ties: lowest bin id)."""
    heap = [(0.0, b) for b in range(nbins)]
    heapq.heapify(heap)
    assign = [0] * len(costs)
    for v in order:
        load, b = heapq.heappop(heap)
        assign[v] = b
        heapq.heappush(heap, (load + costs[v], b))
    return assign


def refine_swap(costs, assign, nbins, tol=0.05, max_iter=None):
    """RefineSwapLB, as read here (the paper gives no constants):

    threshold T = (1 + tol) * mean, mean = total_load(bin loads) / nbins.
    Repeat, at most 4 * nvps times:
      1. Stop if the largest bin load is <= T.
      2. P = most loaded bin (ties: lowest id).
      3. For each other bin Q in order of (load ascending, id ascending):
         a. move: the first VP o of P, in order (cost descending, id
            ascending), with cost > 0 and load(Q) + cost(o) <= T;
            if found, move it and go to 1;
         b. swap: among pairs (o in P, o' in Q) with cost(o) > cost(o'),
            visited in o-order (cost desc, id asc) then o'-order
            (cost asc, id asc), the first pair that minimises
            max(load(P) - d, load(Q) + d) with d = c_o - c_o'; if that value
            is below load(P), swap the two and go to 1.
      4. If no bin Q allowed a move or a swap, stop.
    Loads are kept incrementally: the source's load minus c (a move) or
    minus d (a swap), then the target's load plus the same amount.
    Returns the new assignment (a copy).
    """
    nv = len(costs)
    assign = list(assign)
    loads = bin_loads(costs, assign, nbins)
    thr = (1.0 + tol) * (total_load(loads) / nbins)
    members = [[] for _ in range(nbins)]
    for v, b in enumerate(assign):
        members[b].append(v)
    if max_iter is None:
        max_iter = 4 * nv
    for _ in range(max_iter):
        lmax = max(loads)
        if lmax <= thr:
            break
        P = loads.index(lmax)
        p_order = sorted(members[P], key=lambda v: (-costs[v], v))
        done = False
        for Q in sorted((b for b in range(nbins) if b != P), key=lambda b: (loads[b], b)):
            for o in p_order:
                if costs[o] > 0.0 and loads[Q] + costs[o] <= thr:
                    loads[P] -= costs[o]
                    loads[Q] += costs[o]
                    members[P].remove(o)
                    members[Q].append(o)
                    assign[o] = Q
                    done = True
                    break
            if done:
                break
            q_order = sorted(members[Q], key=lambda v: (costs[v], v))
            best, pair = loads[P], None
            for o in p_order:
                for o2 in q_order:
                    if not costs[o] > costs[o2]:
                        continue
                    d = costs[o] - costs[o2]
                    m = max(loads[P] - d, loads[Q] + d)
                    if m < best:
                        best, pair = m, (o, o2)
            if pair is not None:
                o, o2 = pair
                d = costs[o] - costs[o2]
                loads[P] -= d
                loads[Q] += d
                members[P].remove(o)
                members[Q].append(o)
                members[Q].remove(o2)
                members[P].append(o2)
                assign[o], assign[o2] = Q, P
                done = True
                break
        if not done:
            break
    return assign
