"""Order-of-magnitude checks against the paper's own simulations (Sec. V).

The paper stops each simulation at 100 frame errors and prints the number of frames C that took,
so its frame error rate is about 100 / C: codes A-D (4 x 24, p = 422 .. 1024) at 3.2 dB with 30
iterations, and the LDPCCCs derived from them at 3.1 dB with I = 20 processors.  Its shift values
are not printed, so seeded codes of the same J, L, p stand in; their FER must land within a factor
of 3 of the paper's (both sides carry about 10 % binomial error at 100 errors).  This pins the
channel's Eb/N0 convention, the decoders and the LDPCCC derivation end to end.
"""
import numpy as np
import pytest

import synth
from helpers import read_sections

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FACTOR = 3.0


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_0334_gb300 as p

    p.lib()
    return p


@pytest.mark.parametrize("row", read_sections("paper_frame_counts.txt")["block"], ids=lambda r: r[0])
def test_block_code_fer_matches_paper(pkg, row):
    name, p, C = row
    code = pkg.QCCode(synth.qc_shifts(4, 24, p, seed=7), p)
    r = code.ber_sim(3.2, seed=11, first_frame=0, max_frames=20 * C, target_frame_errors=100, gamma=4096,
                     max_iter=30, early_stop=1)
    assert r["frame_errors"] >= 100, r
    fer, paper = r["frame_errors"] / r["frames"], 100.0 / C
    assert paper / FACTOR <= fer <= paper * FACTOR, (name, fer, paper)


@pytest.mark.parametrize("row", read_sections("paper_frame_counts.txt")["ldpccc"], ids=lambda r: r[0])
def test_ldpccc_fer_matches_paper(pkg, row):
    name, p, C = row
    g, T, I = 256, 64, 20
    cc = pkg.LDPCCC(synth.qc_shifts(4, 24, p, seed=7), p, I, g)
    assert (cc.Lambda, cc.ms) == (4, 3)
    llr = torch.empty((g, T, cc.c), dtype=torch.float32, device="cuda")
    hard = torch.empty((g, T, cc.c), dtype=torch.uint8, device="cuda")
    first, fe, fr = 0, 0, 0
    while fe < 100 and fr < 20 * C:
        pkg.ldpccc_channel(cc.handle, 3.1, 5, first, llr)
        _, n = pkg.ldpccc_decode_window(cc.handle, llr, 30.0, hard, None)
        first += T
        if n:
            fe += int((hard[:, :n].sum(dim=2) > 0).sum().item())
            fr += n * g
    cc.close()
    assert fe >= 100, (fe, fr)
    fer, paper = fe / fr, 100.0 / C
    assert paper / FACTOR <= fer <= paper * FACTOR, (name, fer, paper)
