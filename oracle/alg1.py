"""Plain-Python reading of TRUST's Algorithm 1 and its building blocks.

TEST INFRASTRUCTURE ONLY: only the test suite, the package smoke check and the
benchmark's CPU-baseline / reference arm may import this module.

This is a slow, step-by-step restatement of the paper's method, written from
its text, for small graphs. It exists to pin the pieces the GPU kernels are
built from: the bucketed hash table with an ``atomicAdd``-style slot counter
(Algorithm 1, ``hashTableConstruction``), the linear search inside a bucket
(``linearSearch``), overflow into the next bucket once a bucket reaches its
maximum collision count (Sec. 3.2, last paragraph), the level-major
("interleaved") bucket layout (Sec. 3.2, Fig. linearVsbinary example), the
virtual-combination index map (Sec. 4.2, Fig. combination example) and the
two cost models of Sec. 4.1 (Eq. 1 and Eq. 2).

Readings taken where the paper leaves a choice (each also listed in the design
notes):
* the hash is ``x % B`` (Algorithm 1, ``hash``); a table can be given another
  bucket function instead, which the tests use to pin the multiplicative-hash
  collision statistics;
* a full bucket (``len == L``) sends the element to bucket ``(i + 1) % B``,
  and a search continues through successor buckets while the bucket it just
  scanned is full;
* Algorithm 1 is run on the oriented graph N+ (no division by 6).
"""
from __future__ import annotations

import bisect


class BucketTable:
    """Hash table of Algorithm 1: B fixed-size buckets of L levels each.

    ``length[i]`` is the bucket's ``len`` field; ``level[j][i]`` is
    ``element(j)`` of bucket i, i.e. the level-major layout in which element
    j of bucket i sits at flat position ``j * B + i``.
    """

    def __init__(self, B: int, L: int, hash_fn=None):
        if B < 1 or L < 1:
            raise ValueError("B and L must be positive")
        self.B = B
        self.L = L
        self.hash_fn = hash_fn          # None: Algorithm 1's x % B; else a callable (x, B) -> bucket
        self.length = [0] * B           # hashTable(i).len = 0 for every i
        self.level = [[None] * B for _ in range(L)]

    def hash(self, x: int) -> int:
        if self.hash_fn is not None:
            return self.hash_fn(x, self.B)
        return x % self.B

    def insert(self, v: int) -> int:
        """Place v; returns the bucket it landed in. The slot is the old value
        of the bucket's counter (the paper's atomicAdd(len, 1))."""
        i = self.hash(v)
        for _ in range(self.B):
            slot = self.length[i]
            if slot < self.L:
                self.length[i] = slot + 1
                self.level[slot][i] = v
                return i
            i = (i + 1) % self.B      # bucket full: next bucket
        raise OverflowError("table full")

    def linear_search(self, w: int) -> int:
        """1 if w is stored, else 0: scan the bucket of w level by level, then
        the following buckets while the scanned bucket was full."""
        i = self.hash(w)
        for _ in range(self.B):
            for j in range(self.length[i]):
                if self.level[j][i] == w:
                    return 1
            if self.length[i] < self.L:
                return 0
            i = (i + 1) % self.B
        return 0

    def flat(self) -> list:
        """Level-major memory image: position j*B + i holds element j of bucket i."""
        return [self.level[j][i] for j in range(self.L) for i in range(self.B)]

    def max_collision(self) -> int:
        return max(self.length) if self.length else 0


def hash_table_construction(neighbor_list, B: int, L: int, hash_fn=None) -> BucketTable:
    t = BucketTable(B, L, hash_fn)
    for v in neighbor_list:
        t.insert(int(v))
    return t


def intersection(table: BucketTable, neighbor_list) -> int:
    return sum(table.linear_search(int(w)) for w in neighbor_list)


def count_alg1(dag_ptr, dag_col, B: int = 32, L: int = 128) -> int:
    """Algorithm 1 on an oriented graph: for every u, build the table of N+(u)
    once and add |table ∩ N+(v)| for every v in N+(u). Needs B*L > d+(u)."""
    total = 0
    n = len(dag_ptr) - 1
    for u in range(n):
        nu = dag_col[dag_ptr[u]:dag_ptr[u + 1]]
        if len(nu) < 2:
            continue        # a vertex needs two out-neighbours to close a triangle (Sec. 4.3)
        t = hash_table_construction(nu, B, L)
        for v in nu:
            total += intersection(t, dag_col[dag_ptr[v]:dag_ptr[v + 1]])
    return total


def inclusive_prefix(degrees) -> list:
    out, acc = [], 0
    for d in degrees:
        acc += int(d)
        out.append(acc)
    return out


def vc_locate(prefix_inclusive, k: int):
    """Virtual combination (Sec. 4.2): flat index k of the combined 2-hop list
    -> (j, offset): the j-th out-neighbour's list holds index k, at that offset.
    """
    j = bisect.bisect_right(prefix_inclusive, k)
    start = prefix_inclusive[j - 1] if j > 0 else 0
    return j, k - start


def collective_degree(dag_ptr, dag_col, u: int) -> int:
    """sum over v in N(u) of degree(v) (Eq. 2, here on the oriented graph)."""
    return sum(dag_ptr[v + 1] - dag_ptr[v] for v in dag_col[dag_ptr[u]:dag_ptr[u + 1]])


def cost_eq1(dag_ptr, dag_col, B: int, L: int) -> int:
    """Eq. 1: sum_u sum_{v in N(u)} sum_{w in N(v)} len(bucket of w in HT_u)."""
    c = 0
    for u in range(len(dag_ptr) - 1):
        nu = dag_col[dag_ptr[u]:dag_ptr[u + 1]]
        if not len(nu):
            continue
        t = hash_table_construction(nu, B, L)
        for v in nu:
            for w in dag_col[dag_ptr[v]:dag_ptr[v + 1]]:
                c += t.length[t.hash(int(w))]
    return c


def phi_eq2(dag_ptr, dag_col, B: int, L: int, hash_fn=None) -> int:
    """Eq. 2: sum_u collective_degree(u) * max collision of HT_u (tables built
    with Algorithm 1's hash, or with hash_fn)."""
    phi = 0
    for u in range(len(dag_ptr) - 1):
        nu = dag_col[dag_ptr[u]:dag_ptr[u + 1]]
        if not len(nu):
            continue
        t = hash_table_construction(nu, B, L, hash_fn)
        phi += collective_degree(dag_ptr, dag_col, u) * t.max_collision()
    return phi
