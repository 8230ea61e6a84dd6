"""The proposer's training targets (paper_2012_10684_gb300.proposer.soft_targets),
on the CPU, against the oracle: for each of 64 generated volumes, labelled
with the oracle's threshold, the target is uniform over exactly the
thresholds that give the labelled partition (the oracle's objective is the
same at each of them and the partition changes at the end of the support),
and rows without a threshold are zero."""
import numpy as np
import torch

import oracle
import phantom
from paper_2012_10684_gb300.proposer import soft_targets


def test_soft_targets_cover_the_oracle_partition():
    rng = np.random.default_rng(11)
    hs, ts = [], []
    for i in range(64):
        spec = phantom.chest_volume(1100 + i, 32, 32, int(rng.integers(2, 6)), generations=int(rng.integers(4, 9)),
                                    noise_sd=int(rng.integers(5, 31)), vol_id=i)
        h = oracle.hist1d(phantom.generate_host(spec))
        t, _, _, _, _ = oracle.search1d(h, float(np.float32(0.8)))
        hs.append(h)
        ts.append(t)
    hs.append(np.zeros(4096, np.int64))   # an empty histogram: no threshold
    ts.append(-1)
    H = np.stack(hs)
    y = soft_targets(torch.from_numpy(H.astype(np.int32)), torch.tensor(ts, dtype=torch.int32)).numpy()
    for i, (h, t) in enumerate(zip(hs, ts)):
        if t < 0:
            assert not y[i].any(), i
            continue
        sup = np.nonzero(y[i])[0]
        assert abs(y[i].sum() - 1.0) < 1e-6, i
        assert sup[0] == t and np.all(np.diff(sup) == 1), i
        # the support ends at the next non-empty level (or the last level)
        nxt = np.nonzero(h[t + 1:])[0]
        end = t + 1 + nxt[0] if len(nxt) else 4095
        assert sup[-1] == end - 1, (i, sup[-1], end)
        phi, valid = oracle.objective1d(h, float(np.float32(0.8)))
        inside = [s for s in sup if s < len(phi) and valid[s]]
        assert all(phi[s] == phi[t] for s in inside), i
