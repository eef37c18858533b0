"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and map its permuted outputs back to particle ids."""
import numpy as np

from paper_2206_11998_gb300 import lp


def ensure_built():
    from paper_2206_11998_gb300 import build
    build.build()


def gpu_neighbor_ids(ctx, ps):
    """(ids in GPU order, list of neighbour-id arrays, totals, d2min, keys)."""
    n = ps.n
    cnt, tot, idx, d2, keys = ctx.export_neighbors(n)
    cnt = cnt.cpu().numpy()
    idx = idx.cpu().numpy()
    ids = ps.id.cpu().numpy().astype(np.int64)
    lists = [ids[idx[i, :cnt[i]]] for i in range(n)]
    return ids, lists, tot.cpu().numpy(), d2.cpu().numpy(), keys.cpu().numpy().view(np.uint64)


def by_id(ids, arr):
    """Reorder a per-particle array from GPU order to id order."""
    out = np.empty_like(arr)
    out[ids] = arr
    return out


def normwise(g, o):
    """max |g - o| / max |o| (per-field normwise relative error)."""
    den = np.abs(o).max()
    num = np.abs(g - o).max()
    return num / den if den > 0 else num


def state_by_id(ps, n_fluid):
    st = ps.to_state(n_fluid)
    ids = st["id"].astype(np.int64)
    out = {"x": [by_id(ids, a) for a in st["x"]], "V": by_id(ids, st["V"]), "u": [by_id(ids, a) for a in st["u"]],
           "P": by_id(ids, st["P"]), "m": by_id(ids, st["m"]), "id": np.arange(len(ids), dtype=np.uint32),
           "n_fluid": n_fluid}
    return out
