"""Resumable solves through libmsp: the class pieces of a checkpointed solve
give the oracle's solution set, also after an interrupted first run."""
import pytest

import msp_instances as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as m
    return m


# (5,40): 2^7 classes on the direct pass, 2^4 set for the streaming pass, so
# that each of the 8 pieces holds classes
@pytest.mark.parametrize("plan", [{"direct": 1}, {"direct": 0, "class_bits": 4}], ids=["direct", "streaming"])
def test_resumed_solve_equals_oracle(msp, plan, tmp_path):
    from paper_2507_05045_gb300 import checkpoint
    A, d, x = mi.generate(5, 40, 540, planted=True, h=20)
    want = oracle.mitm(A, d)
    assert mi.mask_of(x) in want

    def interrupted(A, d, class_part=None, **kw):
        # the process is lost before piece 3 runs (a host-side exception)
        if class_part[0] == 3:
            raise RuntimeError("interrupted")
        return msp.Instance(A, d, class_part=class_part, **kw)

    path = str(tmp_path / "ck.json")
    with pytest.raises(RuntimeError):
        checkpoint.solve_resumable(A, d, path, parts=8, plan=plan, instance=interrupted)
    got = checkpoint.solve_resumable(A, d, path, parts=8, plan=plan)
    assert got == want
