"""The hash ceiling helper computes SplitMix64 chains exactly (checked against the oracle's
mixer on sampled threads)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_mix64_burn_values(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    dmx.load()
    out = dmx.dm_mix64_burn(3, 5, seed=77).cpu().numpy().view(np.uint64)
    for tid in (0, 1, 255, 256, 767):
        st = [(77 + tid) & (2 ** 64 - 1)]
        st += [st[0] ^ 0x1111111111111111, st[0] ^ 0x2222222222222222, st[0] ^ 0x3333333333333333]
        for _ in range(5):
            st = [oracle_mod.mix64(v) for v in st]
        assert int(out[tid]) == st[0] ^ st[1] ^ st[2] ^ st[3]
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_mix64_burn(3, 0)
