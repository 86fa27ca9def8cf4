"""Scanning without allocating: tid_match_noalloc against the CPU oracle.

tid_match_noalloc is for callers that may not allocate device memory when
they scan -- a server that handed all free device memory to its own pool at
start-up, or a latency-critical loop that cannot afford an allocation's
implicit synchronisation.  Such a caller passes every buffer itself; the
scan's small scratch lives in a fixed array inside the library, shared by all
calls.  Its results must be exactly the oracle's ascending lists (integer
results: no tolerance), also on consecutive calls that reuse that array.

This file is named to be collected last, so a run that stops at its first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["tiny", "university"])
def test_noalloc_equals_oracle_on_consecutive_calls(which, orc):
    from paper_1807_01409_gb300 import build
    build.build()
    st = synth.tiny_store() if which == "tiny" else synth.university_store(2_000_003)
    cols = [torch.from_numpy(c).cuda() for c in (st.s, st.p, st.o)]
    if which == "tiny":
        pats = [q for q in synth.tiny_queries(st)]
    else:
        pats = [q for q, _, _ in synth.university_queries(st)][:12]
    pats.append(synth.Pattern(0, 0, 0))
    want = [orc.match(st.s, st.p, st.o, p.key()) for p in pats]
    stream = torch.cuda.Stream()
    n = st.n
    # buffers come from the caller (here torch); the entry point allocates nothing
    outs = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for _ in range(2)]
    counts = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for a in range(0, len(pats), 2):
        pair = pats[a:a + 2]
        for j, p in enumerate(pair):  # two calls in a row on one stream
            tb.tid_match_noalloc(0, stream.cuda_stream, cols[0], cols[1], cols[2], p, outs[j], counts[j])
        stream.synchronize()
        for j, p in enumerate(pair):
            c = int(counts[j].item())
            w = want[a + j]
            assert c == w.shape[0], (which, p.key(), c, w.shape[0])
            assert np.array_equal(outs[j][:c].cpu().numpy(), w), (which, p.key())


def test_noalloc_cuts_at_capacity(orc):
    """A buffer shorter than the result: the first cap positions are written, the
    buffer past cap is untouched and the count is the full match count."""
    from paper_1807_01409_gb300 import build
    build.build()
    st = synth.university_store(200_003)
    cols = [torch.from_numpy(c).cuda() for c in (st.s, st.p, st.o)]
    key = (0, int(st.p[0]), 0)
    want = orc.match(st.s, st.p, st.o, key)
    assert want.shape[0] > 100
    for cap in (0, 1, 37, want.shape[0] - 1):
        out = torch.full((want.shape[0] + 64,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        tb.tid_match_noalloc(0, None, cols[0], cols[1], cols[2], key, out, cnt, cap=cap)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(cnt.item()) == want.shape[0], cap
        assert np.array_equal(got[:cap], want[:cap]), cap
        assert (got[cap:] == -7).all(), cap


def test_noalloc_store_of_several_segments(orc):
    """A store larger than one launch covers (resident CTAs x chunk, about 239M
    triples on a GB300) is scanned in several launches that continue each
    other's output: counts and lists equal the oracle's, for one- and
    two-column patterns, with results in every segment."""
    from paper_1807_01409_gb300 import build
    build.build()
    n = (1 << 28) + 13
    rng = np.random.default_rng(2024)
    S = rng.integers(1, 1000, n, dtype=np.int32)
    P = rng.integers(1, 5, n, dtype=np.int32)
    dS, dP = torch.from_numpy(S).cuda(), torch.from_numpy(P).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for key in [(int(S[0]), 0, 0), (0, 3, 0), (int(S[-1]), int(P[-1]), 0), (0, 0, int(S[n // 2]))]:
        torch.cuda.synchronize()
        tb.tid_match_noalloc(0, None, dS, dP, dS, key, out, cnt)
        torch.cuda.synchronize()
        want = orc.match(S, P, S, key)
        c = int(cnt.item())
        assert c == want.shape[0], (key, c, want.shape[0])
        assert want[0] < n // 4 and want[-1] > n - n // 4, key  # hits in the first and the last segment
        assert np.array_equal(out[:c].cpu().numpy(), want), key
    del dS, dP, out


def test_noalloc_rejects_bad_arguments():
    from paper_1807_01409_gb300 import build
    build.build()
    x = torch.ones(8, dtype=torch.int32, device="cuda")
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(tb.TidError) as e:
        tb.tid_match_noalloc(0, None, x, x, x, (0, -1, 0), out, cnt)
    assert e.value.code == tb.TID_ERR_ID
    with pytest.raises(tb.TidError) as e:
        tb.tid_match_noalloc(999, None, x, x, x, (0, 1, 0), out, cnt)
    assert e.value.code == tb.TID_ERR_ARG
