"""The committed record of the R-MAT scale-24 certificate run (written by
tests/golden/certify_rmat24_full.py on a GPU host) is whole and says what
the documentation claims: the workload's edge count, the device's edge list
equal to the oracle's, zero violations of the oracle's certificate over
every edge, and a trussness histogram that accounts for every edge."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
RECORD = os.path.join(HERE, "golden", "rmat24_ef16_certificate.txt")


def _read(path):
    rec, hist = {}, {}
    for ln in open(path).read().splitlines():
        if not ln or ln.startswith("#"):
            continue
        f = ln.split()
        if f[0] == "hist":
            hist[int(f[1])] = int(f[2])
        else:
            rec.update(zip(f[0::2], f[1::2]))  # "key value" pairs, one or more a line
    return rec, hist


def test_certificate_record_is_complete_and_clean():
    rec, hist = _read(RECORD)
    assert rec["n"] == str(1 << 24)
    assert int(rec["m"]) == 260381693
    assert rec["edge_list_equal_to_oracle"] == "1"
    assert rec["certificate_violations"] == "0" and rec["first_bad_edge"] == "-1"
    assert sum(hist.values()) == int(rec["m"])
    assert max(hist) == int(rec["t_max"]) and min(hist) >= 2
    assert int(rec["cores"]) >= 1 and int(rec["seconds_certificate"]) > 0
