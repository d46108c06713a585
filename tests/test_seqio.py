"""FASTA / FASTQ ingest (the data-format API, Sec. II.C.1): host-side parsing
into the (codes, offsets) arrays the alignment calls take.  No GPU needed."""
import numpy as np
import pytest

from paper_1701_01575_gb300 import build, dsa
from paper_1701_01575_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    dsa.load_library()


def parse(text, alphabet=dsa.ALPHABET_DNA4, flags=0):
    return dsa.read_sequences(data=text.encode() if isinstance(text, str) else text,
                              alphabet=alphabet, flags=flags)


def seqs_of(codes, offsets):
    return [codes[offsets[k]:offsets[k + 1]].tolist() for k in range(len(offsets) - 1)]


def test_fasta_layout_rules():
    text = ("\n\n>r1 first record\r\nACGT\r\nac gt\r\n\n"
            ";a comment line\n>r2\n>r3\tthird\nTTTT\nuuu\n>r4\nG")   # r2 empty; no final newline
    codes, offsets, names, lines = parse(text)
    assert seqs_of(codes, offsets) == [[0, 1, 2, 3, 0, 1, 2, 3], [], [3] * 7, [2]]
    assert names == ["r1 first record", "r2", "r3\tthird", "r4"]
    assert lines.tolist() == [3, 8, 9, 12]
    codes, offsets, names, _ = parse(text, flags=dsa.READ_SKIP_EMPTY)
    assert names == ["r1 first record", "r3\tthird", "r4"]
    assert offsets.tolist() == [0, 8, 15, 16]


def test_fastq_records_and_quality_rules():
    text = ("@q1\nACGT\n+\nIIII\n"
            "@q2 multi\nAC\nGT\nA\n+q2 multi\n@II\n+I\n"         # qualities start with '@' and '+'
            ">f1\nCC\n"                                           # FASTA after FASTQ
            "@q3\n\n+\n\n")                                       # empty FASTQ record
    codes, offsets, names, lines = parse(text)
    assert seqs_of(codes, offsets) == [[0, 1, 2, 3], [0, 1, 2, 3, 0], [1, 1], []]
    assert names == ["q1", "q2 multi", "f1", "q3"]
    assert lines.tolist() == [1, 5, 12, 14]


@pytest.mark.parametrize("text,msg", [
    ("ACGT\n", "line 1: a record must start"),
    (">a\nACGN\n", "line 2: character 'N'"),
    (">a\nAC-T\n", "line 2: character '-'"),
    ("@a\nACGT\nACGT\n", "FASTQ record has no '+' line"),
    ("@a\nACGT\n+\nIII\n", "FASTQ quality shorter"),
    ("@a\nACGT\n+\nIIIII\n", "line 4: FASTQ quality longer"),
])
def test_errors_name_the_line(text, msg):
    with pytest.raises(dsa.DsaError) as ex:
        parse(text)
    assert ex.value.code == dsa.ERR_INVALID_ARG and msg in str(ex.value)


def test_error_is_sticky_and_earlier_batches_survive():
    r = dsa.Reader(data=b">a\nAC\n>b\nAXGT\n>c\nGG\n", alphabet=dsa.ALPHABET_DNA4)
    codes, offsets, names, _ = r.next_batch(max_seqs=1)
    assert names == ["a"] and codes.tolist() == [0, 1]
    for _ in range(2):
        with pytest.raises(dsa.DsaError) as ex:
            r.next_batch()
        assert "line 4" in str(ex.value)
    r.close()


def test_alphabets():
    codes, _, _, _ = parse(">a\nACGTURYSWKMBDHVN\n", dsa.ALPHABET_DNA5)
    assert codes.tolist() == [0, 1, 2, 3, 3] + [4] * 11
    codes, _, _, _ = parse(">a\nACGTN-.9\n", dsa.ALPHABET_DNA4, dsa.READ_MAP_UNKNOWN)
    assert codes.tolist() == [0, 1, 2, 3, 0, 0, 0, 0]
    codes, _, _, _ = parse(">a\nACGT?\n", dsa.ALPHABET_DNA5, dsa.READ_MAP_UNKNOWN)
    assert codes.tolist() == [0, 1, 2, 3, 4]
    letters = W.PROTEIN_LETTERS
    codes, _, _, _ = parse(">p\n" + letters + letters.lower() + "UOJ\n", dsa.ALPHABET_PROTEIN)
    assert codes.tolist() == list(range(24)) * 2 + [22, 22, 22]
    with pytest.raises(dsa.DsaError):
        parse(">p\nAC#D\n", dsa.ALPHABET_PROTEIN)
    codes, _, _, _ = parse(">p\nAC#D\n", dsa.ALPHABET_PROTEIN, dsa.READ_MAP_UNKNOWN)
    assert codes.tolist() == [0, 4, 22, 3]


def test_bad_arguments():
    with pytest.raises(dsa.DsaError):
        dsa.Reader(data=b">a\nA\n", alphabet=9)
    with pytest.raises(dsa.DsaError):
        dsa.Reader(data=b">a\nA\n", flags=64)
    with pytest.raises(dsa.DsaError) as ex:
        dsa.Reader(path="/nonexistent/file.fa")
    assert "cannot open" in str(ex.value)
    codes, offsets, names, _ = parse(b"")
    assert len(codes) == 0 and offsets.tolist() == [0] and names == []


def write_fasta(path, seqs, letters, width):
    with open(path, "w") as f:
        for k, s in enumerate(seqs):
            f.write(f">seq{k} len={len(s)}\n")
            text = "".join(letters[c] for c in s)
            for x in range(0, len(text), width):
                f.write(text[x:x + width] + "\n")


@pytest.mark.parametrize("chunk", [16, 17, 100, 0])
def test_file_round_trip_with_chunk_boundaries(tmp_path, chunk):
    """Records written as FASTA (60-column lines, some records longer than the
    read chunk) come back as the same codes, whatever the chunk size."""
    rng = np.random.default_rng(chunk)
    seqs = [rng.integers(0, 24, int(n)).astype(np.uint8) for n in rng.integers(1, 400, 60)]
    path = tmp_path / "p.fa"
    write_fasta(path, seqs, W.PROTEIN_LETTERS, 60)
    with dsa.Reader(path=str(path), alphabet=dsa.ALPHABET_PROTEIN, chunk_bytes=chunk) as r:
        codes, offsets, names, _ = r.next_batch()
        assert r.next_batch() is None
    ref = W.SeqSet.from_list(seqs)
    assert np.array_equal(codes, ref.codes) and np.array_equal(offsets, ref.offsets)
    assert names == [f"seq{k} len={len(s)}" for k, s in enumerate(seqs)]


def test_batches_respect_limits_and_concatenate(tmp_path):
    rng = np.random.default_rng(3)
    seqs = [rng.integers(0, 4, int(n)).astype(np.uint8) for n in rng.integers(1, 3000, 500)]
    path = tmp_path / "d.fa"
    write_fasta(path, seqs, "ACGT", 70)
    ref = W.SeqSet.from_list(seqs)
    for max_res, max_seqs in [(10_000, 0), (1, 0), (0, 7), (5_000, 3), (10**9, 0)]:
        got_codes, got_lens, n_batches = [], [], 0
        with dsa.Reader(path=str(path), chunk_bytes=4096) as r:
            for codes, offsets, names, _ in r.batches(max_res, max_seqs):
                n = len(offsets) - 1
                assert n >= 1
                if max_seqs:
                    assert n <= max_seqs
                if max_res and n > 1:
                    assert offsets[-1] <= max_res
                got_codes.append(codes)
                got_lens.extend(np.diff(offsets).tolist())
                n_batches += 1
        assert np.array_equal(np.concatenate(got_codes), ref.codes)
        assert got_lens == ref.lengths.tolist()
        if max_res == 1:
            assert n_batches == len(seqs)
