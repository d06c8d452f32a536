"""Sample-sharded evaluation over several GPUs (one process per GPU).

The population's fitness (Sec. 1: accuracy, here exact correct counts) is a sum over samples, and
the paper's parallel evaluation (Sec. 3) treats every sample independently. Partitioned by sample
ranges, each rank registers only its own rows, evaluates every rule set of the population on them
with the library's kernels, and one exchange step combines the results:

  hard   correct[P] and per_class[P][K] are int32 sums: one all-reduce (SUM), exact and
         independent of the reduction order;
  soft   the mean loss and its gradients are sums over samples weighted by N_r / N: each rank
         evaluates its shard with dloss scaled by N_r / N, and the per-rank results are gathered
         and added in rank order, so the float sums are the same on every rank and run to run.

Data never crosses ranks: each rank reads its own rows (host or its own device) and the
collectives carry only the P (and P x K, or 3 x C) results. The process group is a
torch.distributed group (NCCL between GPUs; gloo on hosts without CUDA, where `evaluate` must be
given, since the library's kernels need a GPU).
"""
from __future__ import annotations

import numpy as np


def sample_ranges(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, disjoint [start, stop) ranges covering 0..N-1, sizes differing by at most one
    (the first N % world ranges one longer)."""
    if world < 1 or N < 0:
        raise ValueError("world >= 1 and N >= 0 required")
    base, extra = divmod(N, world)
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


class SampleShard:
    """This rank's share of a dataset.

    X, y: the whole dataset's rows (only this rank's range is read and registered), or only this
    rank's rows when `local_rows` is True (then N is the total sample count over all ranks).
    evaluate: optional `(X_shard, y_shard, K, batch) -> (correct, per_class)` used instead of the
    library (CPU ranks in tests); soft_evaluate likewise `(X_shard, y_shard, K, batch, tau,
    dloss) -> dict(loss, grad_a, grad_b, grad_t)`.
    """

    def __init__(self, X, y, K: int, rank: int, world: int, ctx=None, group=None, N: int | None = None,
                 local_rows: bool = False, evaluate=None, soft_evaluate=None):
        self.rank, self.world, self.K = rank, world, K
        self.group = group
        self.ctx = ctx
        self.evaluate = evaluate
        self.soft_evaluate = soft_evaluate
        if local_rows:
            if N is None:
                raise ValueError("local_rows needs the total sample count N")
            self.N = int(N)
            self.X, self.y = X, y
            self.start, self.stop = None, None
        else:
            self.N = int(len(X))
            self.start, self.stop = sample_ranges(self.N, world)[rank]
            self.X, self.y = X[self.start:self.stop], y[self.start:self.stop]
        self.n_local = int(len(self.X))
        self.ds = None
        if ctx is not None and evaluate is None and self.n_local > 0:
            self.ds = ctx.dataset(self.X, self.y, K)

    def close(self):
        if self.ds is not None and self.ctx is not None:
            self.ctx.dataset_destroy(self.ds)
            self.ds = None

    # ------------------------------------------------------------------ collectives
    def _all_reduce_sum(self, t):
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def _gather_in_order(self, t):
        """[world, ...] stack of every rank's tensor, indexed by rank."""
        import torch
        if self.world == 1:
            return t.unsqueeze(0)
        import torch.distributed as dist
        parts = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(parts, t, group=self.group)
        return torch.stack(parts)

    # ------------------------------------------------------------------ hard
    def eval_hard(self, batch, stream=None):
        """Exact correct[P] and per_class[P, K] over all ranks' samples (torch int32 tensors on
        this rank's device, or CPU tensors for CPU ranks)."""
        P, K = batch.P, self.K
        total = self._all_reduce_sum(self.local_hard(batch, stream))
        return total[:P], total[P:].view(P, K)

    def local_hard(self, batch, stream=None):
        """This rank's counts, correct[P] then per_class[P * K], in one int32 tensor."""
        import torch
        P, K = batch.P, self.K
        if self.evaluate is not None:
            c, pc = self.evaluate(self.X, self.y, K, batch)
            local = torch.from_numpy(np.concatenate([np.asarray(c, np.int32).ravel(),
                                                     np.asarray(pc, np.int32).ravel()]))
        elif self.n_local == 0:
            local = torch.zeros(P + P * K, dtype=torch.int32, device=torch.device("cuda"))
        else:
            from . import rs
            db = batch if isinstance(batch, rs.DeviceBatch) else rs.DeviceBatch.from_host(batch)
            dev = db.t["set_default"].device
            local = torch.empty(P + P * K, dtype=torch.int32, device=dev)
            out = (local[:P], local[P:].view(P, K), None)
            self.ctx.eval_hard(self.ds, db, K, out=out, stream=stream)
            if stream is not None:
                stream.synchronize()
        return local

    # ------------------------------------------------------------------ soft
    def soft(self, batch, tau: float, dloss):
        """Mean loss over all N samples and its gradients w.r.t. every condition's a, b, t (as the
        whole-dataset rs_eval_soft_bwd would give them), summed over ranks in rank order."""
        stacked = self._gather_in_order(self.local_soft(batch, tau, dloss))
        total = stacked[0].clone()
        for r in range(1, self.world):            # fixed order: the same sum on every rank
            total += stacked[r]
        P, C = batch.P, batch.C
        return {"loss": total[:P], "grad_a": total[P:P + C], "grad_b": total[P + C:P + 2 * C],
                "grad_t": total[P + 2 * C:]}

    def local_soft(self, batch, tau: float, dloss):
        """This rank's share: loss[P] x N_r / N, then the gradients [3 C] of dloss x N_r / N
        times its shard's mean loss, in one tensor."""
        import torch
        w = self.n_local / self.N
        dl = np.asarray(dloss, np.float64) * w
        if self.soft_evaluate is not None:
            r = self.soft_evaluate(self.X, self.y, self.K, batch, tau, dl)
            parts = [np.asarray(r["loss"], np.float64) * w, r["grad_a"], r["grad_b"], r["grad_t"]]
            local = torch.from_numpy(np.concatenate([np.asarray(p, np.float64).ravel() for p in parts]))
        else:
            from . import rs
            db = batch if isinstance(batch, rs.DeviceBatch) else rs.DeviceBatch.from_host(batch)
            dev = db.t["set_default"].device
            if self.n_local == 0:
                local = torch.zeros(batch.P + 3 * batch.C, dtype=torch.float32, device=dev)
            else:
                ga, gb, gt, loss = self.ctx.soft_bwd(self.ds, db, tau,
                                                     torch.tensor(dl, dtype=torch.float32, device=dev))
                local = torch.cat([loss * w, ga, gb, gt])
        return local
