"""Index persistence (gn_index_save / gn_index_load): a loaded index is the saved one.

The paper keeps its inverted index on disk and loads it when the service starts
("Inverted Indexes" section).  A loaded index must export the same buckets and
occurrences and give identical search results; damaged or foreign files are
rejected with GN_EINVAL."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("stride,mask", [(11, None), (1, None), (18, "111010010100110111")])
def test_saved_index_searches_the_same(gn, tmp_path, stride, mask):
    bank = synth.make_bank("mid", n_seqs=5000)
    qs = synth.make_queries("mid", bank, n=40)
    ix = gn.Index.from_bank(bank, stride=stride, mask=mask)
    path = str(tmp_path / f"mid_s{stride}.gnidx")
    ix.save(path)
    assert os.path.getsize(path) > 0
    ld = gn.Index.load(path)
    a, b = ix.info(), ld.info()
    assert (a.k, a.stride, a.n_seqs, a.n_bases, a.n_postings) == (b.k, b.stride, b.n_seqs, b.n_bases, b.n_postings)
    for x, y in zip(ix.export(), ld.export()):
        assert np.array_equal(x, y)
    r1 = gn.search(ix, qs.start, qs.bases).all()
    r2 = gn.search(ld, qs.start, qs.bases).all()
    assert sum(len(r) for r in r1) > 0
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)
    ld.close()
    ix.close()


def test_bad_files_rejected(gn, tmp_path):
    bank = synth.make_bank("tiny", n_seqs=200)
    ix = gn.Index.from_bank(bank)
    good = str(tmp_path / "tiny.gnidx")
    ix.save(good)
    data = open(good, "rb").read()
    cases = {"missing": None, "not_index": b"hello world" * 20, "truncated": data[: len(data) // 2],
             "bad_version": data[:8] + (99).to_bytes(8, "little") + data[16:]}
    for name, content in cases.items():
        p = str(tmp_path / f"{name}.gnidx")
        if content is not None:
            open(p, "wb").write(content)
        with pytest.raises(gn.GnError) as e:
            gn.Index.load(p)
        assert e.value.status == gn.GN_EINVAL, name
    with pytest.raises(gn.GnError) as e:
        ix.save(str(tmp_path / "no_such_dir" / "x.gnidx"))
    assert e.value.status == gn.GN_EINVAL
    ix.close()
