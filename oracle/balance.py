"""Balancer oracle (TEST INFRASTRUCTURE ONLY): plain-Python restatements of
the two Charm++ strategies the paper uses (Sec. VI) and of the initial
block placement.

The balancers compare loads on a fixed-point grid (`fixed_point`): every
cost is rounded once to an integer multiple of 2^-e, with e chosen so that
every load and every total is an integer below 2^53.  Sums are then exact in
any order and exactly representable in FP64, so any implementation that
rounds the costs the same way reproduces these assignments bit for bit,
whatever order it adds in.

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
  greedy_blocked -- GreedyLB applied to consecutive blocks of nbins objects
                    of a given order: within a block the heaviest object
                    goes to the least loaded processor, the next heaviest to
                    the next, ... (one object per processor per block).
"""
import heapq
import math


def static_blocks(nvps, nbins):
    """VP v goes to bin floor(v * nbins / nvps): contiguous, sizes differ by <= 1."""
    return [(v * nbins) // nvps for v in range(nvps)]


def bin_loads(costs, assign, nbins):
    """Per-bin sum of the given costs, VPs added in increasing id order."""
    loads = [0] * nbins
    for v, b in enumerate(assign):
        loads[b] += costs[v]
    return loads


def fixed_point(costs):
    """The costs (FP64, >= 0) as integers on the balancers' grid:
    q_v = c_v * 2^e rounded to the nearest integer (ties to even), where
    e = 53 - L - x, L = bit length of the VP count and 2^(x-1) <= max c < 2^x.
    The largest cost then lies in [2^(52-L), 2^(53-L)], so the sum of all
    costs stays below 2^53.  All zero when every cost is zero."""
    n = len(costs)
    cmax = max(costs) if n else 0.0
    if not cmax > 0.0:
        return [0] * n
    _, x = math.frexp(cmax)
    e = 53 - n.bit_length() - x
    return [round(math.ldexp(c, e)) for c in costs]


def max_over_mean(costs, assign, nbins):
    """Largest bin load over the mean load, on the fixed-point grid:
    float(max load) / (float(total) / nbins)."""
    q = fixed_point(costs)
    loads = bin_loads(q, assign, nbins)
    mean = float(sum(q)) / nbins
    return float(max(loads)) / mean if mean > 0 else 1.0


def migrations(old, new):
    return sum(1 for a, b in zip(old, new) if a != b)


def greedy(costs, nbins):
    """GreedyLB.  Order VPs by (cost descending, id ascending); give each in
    turn to the bin with the least load so far (ties: lowest bin id); costs
    and loads on the fixed-point grid."""
    q = fixed_point(costs)
    order = sorted(range(len(q)), key=lambda v: (-q[v], v))
    return _list_schedule(q, nbins, order)


def greedy_ordered(costs, nbins, order):
    """Objects in the given order (a permutation of VP ids), each to the bin
    with the least load so far (ties: lowest bin id)."""
    return _list_schedule(fixed_point(costs), nbins, order)


def greedy_blocked(costs, nbins, order):
    """Objects in the given order, in consecutive blocks of nbins: within a
    block, objects by (cost descending, id ascending) go to the bins by
    (load ascending, id ascending), one each; loads on the fixed-point grid.
    A short last block fills the least loaded bins."""
    q = fixed_point(costs)
    loads = [0] * nbins
    assign = [0] * len(q)
    for base in range(0, len(order), nbins):
        block = sorted(order[base:base + nbins], key=lambda v: (-q[v], v))
        bins = sorted(range(nbins), key=lambda b: (loads[b], b))
        for v, b in zip(block, bins):
            assign[v] = b
            loads[b] += q[v]
    return assign


def _list_schedule(q, nbins, order):
    heap = [(0, b) for b in range(nbins)]
    heapq.heapify(heap)
    assign = [0] * len(q)
    for v in order:
        load, b = heapq.heappop(heap)
        assign[v] = b
        heapq.heappush(heap, (load + q[v], b))
    return assign


def refine_swap(costs, assign, nbins, tol=0.05, max_iter=None):
    """RefineSwapLB, as read here (the paper gives no constants); costs and
    loads on the fixed-point grid (q):

    threshold T = (1 + tol) * (float(sum of q) / nbins).
    Repeat, at most 4 * nvps times:
      1. Stop if the largest bin load is <= T.
      2. P = most loaded bin (ties: lowest id).
      3. For each other bin Q in order of (load ascending, id ascending):
         a. move: the first VP o of P, in order (cost descending, id
            ascending), with q_o > 0 and load(Q) + q_o <= T;
            if found, move it and go to 1;
         b. swap: among pairs (o in P, o' in Q) with q_o > q_o', visited in
            o-order (cost desc, id asc) then o'-order (cost asc, id asc),
            the first pair that minimises max(load(P) - d, load(Q) + d) with
            d = q_o - q_o'; if that value is below load(P), swap the two and
            go to 1.
      4. If no bin Q allowed a move or a swap, stop.
    Returns the new assignment (a copy).
    """
    q = fixed_point(costs)
    nv = len(q)
    assign = list(assign)
    loads = bin_loads(q, assign, nbins)
    thr = (1.0 + tol) * (float(sum(q)) / nbins)
    members = [[] for _ in range(nbins)]
    for v, b in enumerate(assign):
        members[b].append(v)
    if max_iter is None:
        max_iter = 4 * nv
    for _ in range(max_iter):
        lmax = max(loads)
        if float(lmax) <= thr:
            break
        P = loads.index(lmax)
        p_order = sorted(members[P], key=lambda v: (-q[v], v))
        done = False
        for Q in sorted((b for b in range(nbins) if b != P), key=lambda b: (loads[b], b)):
            for o in p_order:
                if q[o] > 0 and float(loads[Q] + q[o]) <= thr:
                    loads[P] -= q[o]
                    loads[Q] += q[o]
                    members[P].remove(o)
                    members[Q].append(o)
                    assign[o] = Q
                    done = True
                    break
            if done:
                break
            q_order = sorted(members[Q], key=lambda v: (q[v], v))
            best, pair = loads[P], None
            for o in p_order:
                for o2 in q_order:
                    if not q[o] > q[o2]:
                        continue
                    d = q[o] - q[o2]
                    m = max(loads[P] - d, loads[Q] + d)
                    if m < best:
                        best, pair = m, (o, o2)
            if pair is not None:
                o, o2 = pair
                d = q[o] - q[o2]
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
