"""Operation counts used for throughput reporting.

The paper's cost metric for a CCSD run is C = O^2 V^4 (O correlated occupied,
V correlated virtual spinors), the count of its costliest contraction, the
particle-particle ladder (Sec. "Uranyl tris-nitrate", definition of C).

Throughput is reported with 8 real flops per complex multiply-add (4M count).
The ladder's algorithmic count uses the antisymmetry-packed sums
(sum over c<d, i<j, a<b), the dense count 8 O^2 V^4 is reported beside it.
"""


def cost_metric(o: int, v: int) -> int:
    """C = O^2 V^4."""
    return o * o * v ** 4


def pairs(n: int) -> int:
    return n * (n - 1) // 2


def ladder_flops_packed(o: int, v: int) -> int:
    """8 [o(o-1)/2] [v(v-1)/2]^2: complex GEMM (ij pairs) x (cd pairs) x (ab pairs)."""
    return 8 * pairs(o) * pairs(v) ** 2


def df_default_block(v: int) -> int:
    """Rows a per rebuilt block of (ac|bd) when <ab||cd> is not stored (about 6 GB of D)."""
    return max(1, min(int(6e9 / (16.0 * v ** 3)), max(v - 1, 1)))


def df_rebuild_cmacs(v: int, naux: int, blk: int = 0) -> float:
    """Complex multiply-adds of the (ac|bd) rebuild over Q: one GEMM per block a in [a0, a1)
    of M = (a1 - a0) v rows (a, c), N = (v - a0 - 1) v columns (b > a0, d), K = naux."""
    blk = blk or df_default_block(v)
    total = 0.0
    for a0 in range(0, v - 1, blk):
        a1 = min(v - 1, a0 + blk)
        total += float(a1 - a0) * v * float(v - a0 - 1) * v * naux
    return total


def ladder_flops_dense(o: int, v: int) -> int:
    """8 o^2 v^4 (= 8 C)."""
    return 8 * cost_metric(o, v)


def ring_flops(o: int, v: int) -> int:
    """8 (ov)^3: the ring GEMM (ai) x (ck) x (bj)."""
    return 8 * (o * v) ** 3


def triples_cmacs(o: int, v: int) -> dict:
    """Complex multiply-adds of the triples GEMMs over all i<j<k: the three e-terms form
    [v(v-1)/2] x v outputs over K = v, the three m-terms v x [v(v-1)/2] over K = o."""
    nt = o * (o - 1) * (o - 2) // 6
    pv = pairs(v)
    return {"e": 3.0 * nt * pv * v * v, "m": 3.0 * nt * v * pv * o}
