"""Python face of the C ABI, over torch device tensors.

Every function here only checks shapes, takes ``data_ptr()`` and the current
CUDA stream, and calls the native library; all arithmetic runs in the CUDA
kernels.  Multi-precision arrays are held in int32 tensors whose bits are the
uint32 limbs (little-endian limbs, one row per value); uint64 values are held
in int64 tensors.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native
from .native import call, lib


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor) -> int:
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _limbs_from_int(x: int, limbs: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(4 * limbs, "little"), dtype="<u4").copy()


def _int_from_limbs(a) -> int:
    return int.from_bytes(np.asarray(a, dtype="<u4").tobytes(), "little")


class Key:
    """A Paillier key held by the library (private: p, q; public: n)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)
        self.n_bits = lib().paillier_key_bits(self._h)
        self.L = self.n_bits // 32
        self.is_private = bool(lib().paillier_key_is_private(self._h))

    @property
    def handle(self):
        return self._h

    @classmethod
    def generate(cls, n_bits: int, seed: int) -> "Key":
        out = C.c_void_p()
        call("paillier_keygen", n_bits, C.c_uint64(seed), C.byref(out))
        return cls(out.value)

    @classmethod
    def from_primes(cls, n_bits: int, p: int, q: int) -> "Key":
        lh = n_bits // 64
        pa, qa = _limbs_from_int(p, lh), _limbs_from_int(q, lh)
        out = C.c_void_p()
        call("paillier_key_import", n_bits, pa.ctypes.data, qa.ctypes.data, C.byref(out))
        return cls(out.value)

    @classmethod
    def public(cls, n_bits: int, n: int) -> "Key":
        na = _limbs_from_int(n, n_bits // 32)
        out = C.c_void_p()
        call("paillier_key_import_public", n_bits, na.ctypes.data, C.byref(out))
        return cls(out.value)

    def export(self):
        """(n, p, q) as Python ints (p, q None for a public key)."""
        na = np.zeros(self.L, dtype=np.uint32)
        if self.is_private:
            pa = np.zeros(self.L // 2, dtype=np.uint32)
            qa = np.zeros(self.L // 2, dtype=np.uint32)
            call("paillier_key_export", self._h, na.ctypes.data, pa.ctypes.data, qa.ctypes.data)
            return _int_from_limbs(na), _int_from_limbs(pa), _int_from_limbs(qa)
        call("paillier_key_export", self._h, na.ctypes.data, None, None)
        return _int_from_limbs(na), None, None

    def close(self):
        if self._h is not None and self._h.value:
            lib().paillier_key_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode(v: torch.Tensor, stream=None) -> torch.Tensor:
    """Fixed-point plaintexts of float32 values (int64 tensor of uint64 bits)."""
    assert v.dtype == torch.float32
    out = torch.empty(v.shape, dtype=torch.int64, device=v.device)
    call("paillier_encode", _ptr(v), v.numel(), _ptr(out), _stream(stream))
    return out


def decode(s: torch.Tensor, cnt: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Float64 values of fixed-point sums s (int64 bits) of cnt encoded values each."""
    assert s.dtype == torch.int64 and cnt.dtype == torch.int32 and s.numel() == cnt.numel()
    if out is None:
        out = torch.empty(s.shape, dtype=torch.float64, device=s.device)
    call("paillier_decode", _ptr(s), _ptr(cnt), s.numel(), _ptr(out), _stream(stream))
    return out


def encrypt(key: Key, m: torch.Tensor, r: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Ciphertexts [count, 2L] (int32 bits) of plaintexts m [count] (int64 bits)
    under randomness r [count, L] (int32 bits)."""
    count = m.numel()
    assert m.dtype == torch.int64 and r.dtype == torch.int32 and r.shape == (count, key.L)
    if out is None:
        out = torch.empty((count, 2 * key.L), dtype=torch.int32, device=m.device)
    call("paillier_encrypt", key.handle, _ptr(m), _ptr(r), count, _ptr(out), _stream(stream))
    return out


def ct_prepare(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Montgomery form (mod n^2) of ciphertexts [..., 2L]."""
    assert ct.dtype == torch.int32 and ct.shape[-1] == 2 * key.L
    count = ct.numel() // (2 * key.L)
    if out is None:
        out = torch.empty_like(ct)
    call("paillier_ct_prepare", key.handle, _ptr(ct), count, _ptr(out), _stream(stream))
    return out


def hist_aggregate(key: Key, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int, K: int,
                   hist: torch.Tensor | None = None, count: torch.Tensor | None = None, per_node: bool = False,
                   stream=None):
    """Encrypted histogram [num_nodes, F, K, 2, 2L] and counts [num_nodes, F, K]
    from Montgomery-form ciphertexts ctm [2, M, 2L], bins [F, M] uint8, node [M] int32."""
    M = node.numel()
    F = bins.shape[0]
    assert ctm.dtype == torch.int32 and ctm.shape == (2, M, 2 * key.L)
    assert bins.dtype == torch.uint8 and bins.shape == (F, M) and node.dtype == torch.int32
    if hist is None:
        hist = torch.empty((num_nodes, F, K, 2, 2 * key.L), dtype=torch.int32, device=ctm.device)
    if count is None:
        count = torch.empty((num_nodes, F, K), dtype=torch.int32, device=ctm.device)
    fn = "paillier_hist_aggregate_per_node" if per_node else "paillier_hist_aggregate"
    call(fn, key.handle, _ptr(ctm), M, _ptr(bins), F, K, _ptr(node), num_nodes, _ptr(hist), _ptr(count),
         _stream(stream))
    return hist, count


def decrypt(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Plaintexts [count, L] (int32 bits) of ciphertexts [..., 2L]."""
    assert ct.dtype == torch.int32 and ct.shape[-1] == 2 * key.L
    count = ct.numel() // (2 * key.L)
    if out is None:
        out = torch.empty((count, key.L), dtype=torch.int32, device=ct.device)
    call("paillier_decrypt", key.handle, _ptr(ct), count, _ptr(out), _stream(stream))
    return out


def decrypt_u64(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Plaintexts as uint64 (int64 tensor) of ciphertexts [..., 2L]."""
    assert ct.dtype == torch.int32 and ct.shape[-1] == 2 * key.L
    count = ct.numel() // (2 * key.L)
    if out is None:
        out = torch.empty(ct.shape[:-1], dtype=torch.int64, device=ct.device)
    call("paillier_decrypt_u64", key.handle, _ptr(ct), count, _ptr(out), _stream(stream))
    return out


class LevelPlan:
    """Batched tree-level path: one pass over all nodes of a level, captured
    into a CUDA graph on the first run and replayed for later levels.  gh=True:
    one g/h-packed ciphertext array per sample ([M, 2L] in, [nodes, F, K, 2L] out)."""

    def __init__(self, key: Key, M: int, F: int, K: int, max_nodes: int, gh: bool = False):
        out = C.c_void_p()
        fn = "paillier_level_plan_create_gh" if gh else "paillier_level_plan_create"
        call(fn, key.handle, M, F, K, max_nodes, C.byref(out))
        self._h = out
        self.key, self.M, self.F, self.K, self.max_nodes, self.gh = key, M, F, K, max_nodes, gh

    def run(self, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int,
            hist: torch.Tensor | None = None, count: torch.Tensor | None = None, stream=None):
        L = self.key.L
        want = (self.M, 2 * L) if self.gh else (2, self.M, 2 * L)
        assert ctm.shape == want and bins.shape == (self.F, self.M) and node.numel() == self.M
        if hist is None:
            shape = (num_nodes, self.F, self.K, 2 * L) if self.gh else (num_nodes, self.F, self.K, 2, 2 * L)
            hist = torch.empty(shape, dtype=torch.int32, device=ctm.device)
        if count is None:
            count = torch.empty((num_nodes, self.F, self.K), dtype=torch.int32, device=ctm.device)
        call("paillier_level_run", self._h, _ptr(ctm), _ptr(bins), _ptr(node), num_nodes, _ptr(hist), _ptr(count),
             _stream(stream))
        return hist, count

    def stats(self):
        c, r, k = C.c_int(), C.c_int(), C.c_int()
        call("paillier_level_plan_stats", self._h, C.byref(c), C.byref(r), C.byref(k))
        return {"captures": c.value, "replays": r.value, "kernels": k.value}

    def close(self):
        if self._h is not None and self._h.value:
            lib().paillier_level_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (histogram + decryption jobs)."""

    def __init__(self, slots: int, hbm_budget: int):
        out = C.c_void_p()
        call("pl_server_create", slots, hbm_budget, C.byref(out))
        self._h = out
        self._keep = {}

    def submit(self, key: Key, ctm: torch.Tensor, M: int, F: int, K: int, bins: torch.Tensor,
               node: torch.Tensor | None = None, num_nodes: int = 1, gh_stride: int | None = None,
               bins_stride: int | None = None, pack_bits: int = 0, gh_bits: int = 0):
        """Queues a request over the first M samples / F features of resident
        arrays (ctm: g and h arrays gh_stride rows apart, or with gh_bits one
        g/h-packed array); returns (ticket, host sums [num_nodes, F, K, 2]
        uint64 (pinned), host counts [num_nodes, F, K] int32 (pinned))."""
        sums = torch.empty((num_nodes, F, K, 2), dtype=torch.int64).pin_memory()
        counts = torch.empty((num_nodes, F, K), dtype=torch.int32).pin_memory()
        req = native.Request(key.handle.value, _ptr(ctm), gh_stride if gh_stride is not None else M, M, F, K,
                             _ptr(bins), bins_stride if bins_stride is not None else M,
                             _ptr(node) if node is not None else None, num_nodes, sums.data_ptr(), counts.data_ptr(),
                             pack_bits, gh_bits)
        t = C.c_uint64()
        call("pl_server_submit", self._h, C.byref(req), C.byref(t))
        self._keep[t.value] = (sums, counts, ctm, bins, node, key)
        return t.value, sums, counts

    @staticmethod
    def request_bytes(key: Key, ctm: torch.Tensor, M: int, F: int, K: int, bins: torch.Tensor,
                      node: torch.Tensor | None = None, num_nodes: int = 1, pack_bits: int = 0,
                      gh_bits: int = 0) -> int:
        req = native.Request(key.handle.value, _ptr(ctm), M, M, F, K, _ptr(bins), M,
                             _ptr(node) if node is not None else None, num_nodes, 0, 0, pack_bits, gh_bits)
        b = C.c_size_t()
        call("pl_server_request_bytes", C.byref(req), C.byref(b))
        return b.value

    def poll(self, ticket: int):
        st, lat, err = C.c_int(), C.c_double(), C.c_int()
        call("pl_server_poll", self._h, ticket, C.byref(st), C.byref(lat), C.byref(err))
        return st.value, lat.value, err.value

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        st, lat = C.c_int(), C.c_double()
        call("pl_server_wait", self._h, ticket, timeout_ms, C.byref(st), C.byref(lat))
        return st.value, lat.value

    def cancel(self, ticket: int):
        call("pl_server_cancel", self._h, ticket)

    def stats(self):
        a, b, c, d = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        pr, pb = C.c_int(), C.c_size_t()
        call("pl_server_stats", self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(pr), C.byref(pb))
        return {"submitted": a.value, "completed": b.value, "failed": c.value, "cancelled": d.value,
                "peak_running": pr.value, "peak_bytes": pb.value}

    def release(self, ticket: int):
        self._keep.pop(ticket, None)

    def close(self):
        if self._h is not None and self._h.value:
            lib().pl_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_slots(key: Key, slot_bits: int) -> int:
    return lib().paillier_pack_slots(key.handle, slot_bits)


def pack(key: Key, ct: torch.Tensor, slot_bits: int, out: torch.Tensor | None = None, stream=None):
    """Packed ciphertexts [ceil(count / slots), 2L] of cells ct [..., 2L]."""
    assert ct.dtype == torch.int32 and ct.shape[-1] == 2 * key.L
    count = ct.numel() // (2 * key.L)
    slots = pack_slots(key, slot_bits)
    if out is None:
        out = torch.empty(((count + slots - 1) // slots, 2 * key.L), dtype=torch.int32, device=ct.device)
    call("paillier_pack", key.handle, _ptr(ct), count, slot_bits, _ptr(out), _stream(stream))
    return out


def decrypt_packed_u64(key: Key, packed: torch.Tensor, count: int, slot_bits: int,
                       out: torch.Tensor | None = None, stream=None):
    """The `count` cell plaintexts (int64 bits of uint64) of packed ciphertexts."""
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=packed.device)
    call("paillier_decrypt_packed_u64", key.handle, _ptr(packed), count, slot_bits, _ptr(out), _stream(stream))
    return out


# ---- g/h packing: one plaintext per sample (include/paillier_pack.h) --------

def encode_gh(g: torch.Tensor, h: torch.Tensor, B: int, out: torch.Tensor | None = None, stream=None):
    """m = enc(g) + 2^B enc(h): [count, 2] int64 (bits of the two uint64 words)."""
    assert g.dtype == torch.float32 and h.dtype == torch.float32 and g.shape == h.shape
    count = g.numel()
    if out is None:
        out = torch.empty((count, 2), dtype=torch.int64, device=g.device)
    call("paillier_encode_gh", _ptr(g), _ptr(h), count, B, _ptr(out), _stream(stream))
    return out


def encrypt_gh(key: Key, m: torch.Tensor, r: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Ciphertexts [count, 2L] of two-word plaintexts m [count, 2]."""
    assert m.dtype == torch.int64 and m.shape[-1] == 2
    count = m.numel() // 2
    assert r.dtype == torch.int32 and r.numel() == count * key.L
    if out is None:
        out = torch.empty((count, 2 * key.L), dtype=torch.int32, device=m.device)
    call("paillier_encrypt_gh", key.handle, _ptr(m), _ptr(r), count, _ptr(out), _stream(stream))
    return out


def hist_aggregate_gh(key: Key, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int, K: int,
                      hist: torch.Tensor | None = None, count: torch.Tensor | None = None, stream=None):
    """Encrypted histogram [num_nodes, F, K, 2L] and counts of ONE g/h-packed
    Montgomery-form array ctm [M, 2L]."""
    M = node.numel()
    F = bins.shape[0]
    assert ctm.dtype == torch.int32 and ctm.shape == (M, 2 * key.L)
    assert bins.dtype == torch.uint8 and bins.shape == (F, M) and node.dtype == torch.int32
    if hist is None:
        hist = torch.empty((num_nodes, F, K, 2 * key.L), dtype=torch.int32, device=ctm.device)
    if count is None:
        count = torch.empty((num_nodes, F, K), dtype=torch.int32, device=ctm.device)
    call("paillier_hist_aggregate_gh", key.handle, _ptr(ctm), M, _ptr(bins), F, K, _ptr(node), num_nodes,
         _ptr(hist), _ptr(count), _stream(stream))
    return hist, count


def decrypt_gh(key: Key, ct: torch.Tensor, B: int, out: torch.Tensor | None = None, stream=None):
    """(S_g, S_h) [count, 2] (int64 bits of uint64) of g/h-packed cells ct [..., 2L]."""
    assert ct.dtype == torch.int32 and ct.shape[-1] == 2 * key.L
    count = ct.numel() // (2 * key.L)
    if out is None:
        out = torch.empty((count, 2), dtype=torch.int64, device=ct.device)
    call("paillier_decrypt_gh", key.handle, _ptr(ct), count, B, _ptr(out), _stream(stream))
    return out


def decrypt_packed_gh(key: Key, packed: torch.Tensor, cells: int, B: int, out: torch.Tensor | None = None,
                      stream=None):
    """(S_g, S_h) [cells, 2] of g/h-packed cells packed with pack(slot_bits = 2B)."""
    if out is None:
        out = torch.empty((cells, 2), dtype=torch.int64, device=packed.device)
    call("paillier_decrypt_packed_gh", key.handle, _ptr(packed), cells, B, _ptr(out), _stream(stream))
    return out


def split_find(sums: torch.Tensor, counts: torch.Tensor, lam: float = 1.0, gamma: float = 0.0,
               min_child_weight: float = 0.0, stream=None):
    """Best split per node from decrypted sums [nodes, F, K, 2] (int64 bits of
    uint64) and counts [nodes, F, K]: (feature, bin, gain) tensors [nodes]."""
    nodes, F, K, _ = sums.shape
    assert sums.dtype == torch.int64 and counts.dtype == torch.int32 and counts.shape == (nodes, F, K)
    bf = torch.empty(nodes, dtype=torch.int32, device=sums.device)
    bb = torch.empty_like(bf)
    bg = torch.empty(nodes, dtype=torch.float64, device=sums.device)
    call("paillier_split_find", _ptr(sums), _ptr(counts), nodes, F, K, lam, gamma, min_child_weight, _ptr(bf),
         _ptr(bb), _ptr(bg), _stream(stream))
    return bf, bb, bg


def split_apply(bins: torch.Tensor, node: torch.Tensor, best_f: torch.Tensor, best_b: torch.Tensor,
                out: torch.Tensor | None = None, stream=None):
    """Next-level node ids of every sample under the chosen splits."""
    M = node.numel()
    if out is None:
        out = torch.empty_like(node)
    call("paillier_split_apply", _ptr(bins), M, _ptr(node), _ptr(best_f), _ptr(best_b), _ptr(out), _stream(stream))
    return out


def child_select(next_node: torch.Tensor, counts: torch.Tensor, best_f: torch.Tensor, best_b: torch.Tensor,
                 stream=None):
    """(small_right [parents], small_node [M]): which child of every parent is
    smaller, and the node array of parents restricted to those children."""
    nodes, F, K = counts.shape
    M = next_node.numel()
    sr = torch.empty(nodes, dtype=torch.int32, device=counts.device)
    sn = torch.empty_like(next_node)
    call("paillier_child_select", _ptr(next_node), M, _ptr(counts), nodes, F, K, _ptr(best_f), _ptr(best_b),
         _ptr(sr), _ptr(sn), _stream(stream))
    return sr, sn


def child_subtract(parent_sums, parent_counts, small_sums, small_counts, small_right, stream=None):
    """Child-level sums [2 nodes, F, K, 2] and counts [2 nodes, F, K]."""
    nodes, F, K, _ = parent_sums.shape
    cs = torch.empty((2 * nodes, F, K, 2), dtype=torch.int64, device=parent_sums.device)
    cc = torch.empty((2 * nodes, F, K), dtype=torch.int32, device=parent_sums.device)
    call("paillier_child_subtract", _ptr(parent_sums), _ptr(parent_counts), _ptr(small_sums), _ptr(small_counts),
         _ptr(small_right), nodes, F, K, _ptr(cs), _ptr(cc), _stream(stream))
    return cs, cc


def tree_decide(bins_party: torch.Tensor, f_lo: int, tree_f: torch.Tensor, tree_b: torch.Tensor,
                go_right: torch.Tensor, stream=None):
    """One party fills go_right [nodes, M] (uint8) for the tree nodes on its features."""
    F_party, M = bins_party.shape
    call("paillier_tree_decide", _ptr(bins_party), F_party, f_lo, M, _ptr(tree_f), _ptr(tree_b), tree_f.numel(),
         _ptr(go_right), _stream(stream))
    return go_right


def tree_route(go_right: torch.Tensor, tree_f: torch.Tensor, depth: int, stream=None):
    """Level-order index of the node every sample reaches."""
    M = go_right.shape[1]
    leaf = torch.empty(M, dtype=torch.int32, device=go_right.device)
    call("paillier_tree_route", _ptr(go_right), M, _ptr(tree_f), depth, _ptr(leaf), _stream(stream))
    return leaf


def leaf_weights(sums: torch.Tensor, counts: torch.Tensor, lam: float = 1.0, stream=None):
    nodes, F, K, _ = sums.shape
    w = torch.empty(nodes, dtype=torch.float64, device=sums.device)
    call("paillier_leaf_weights", _ptr(sums), _ptr(counts), nodes, F, K, lam, _ptr(w), _stream(stream))
    return w


def get_config(key: Key, op: int):
    la, pa = C.c_int(), C.c_int()
    call("paillier_get_config", key.handle, op, C.byref(la), C.byref(pa))
    return la.value, pa.value


def set_config(key: Key, op: int, lanes: int, param: int):
    call("paillier_set_config", key.handle, op, lanes, param)


def autotune(key: Key, op: int, cache_path: str | None = None, stream=None):
    la, pa = C.c_int(), C.c_int()
    call("paillier_autotune", key.handle, op, cache_path.encode() if cache_path else None, _stream(stream),
         C.byref(la), C.byref(pa))
    return la.value, pa.value


def sync(stream=None) -> int:
    """Synchronise the stream and raise on a device-reported error; returns the raw status word."""
    st = C.c_int(0)
    call("paillier_sync", _stream(stream), C.byref(st))
    return st.value


def to_limb_tensor(arr: np.ndarray, device="cuda") -> torch.Tensor:
    """uint32 numpy limbs -> int32 torch tensor on the device (bit copy)."""
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32)).to(device)


def from_limb_tensor(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)
