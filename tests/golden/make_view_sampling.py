"""Writes view_sampling_sec3b.json: the (k, j, t, phi) list of the view
sampling rule printed in Sec. III-B, t = 1, a, ..., a^n with a = sqrt(2),
n = 5, and phi = 0, b/t, ..., J b/t with b = 72 deg and J the largest integer
with J b/t < 180 deg.  The bound is evaluated exactly: (72 j)^2 < 180^2 2^k,
i.e. 4 j^2 < 25 2^k.  t = 1 keeps a single view (phi = 0), the ASIFT
convention.  Pure Python from the printed rule: no oracle, no CUDA."""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def sampling(n: int = 5):
    views = [{"k": 0, "j": 0, "t": 1.0, "phi_deg": 0.0}]
    for k in range(1, n + 1):
        t = 2.0 ** (k / 2)
        j = 0
        while 4 * j * j < 25 * 2 ** k:
            views.append({"k": k, "j": j, "t": t, "phi_deg": j * 72.0 / t})
            j += 1
    return views


if __name__ == "__main__":
    views = sampling()
    doc = {
        "source": "Sec. III-B sampling rule: t = 1, a, ..., a^n with a = sqrt(2), n = 5; "
                  "phi = 0, b/t, ..., k b/t with b = 72 deg and the largest k such that k b/t < 180 deg "
                  "(the bound evaluated exactly: 4 j^2 < 25 2^k)",
        "reading": "one view at t = 1 (phi = 0), the ASIFT convention",
        "counts_per_tilt": {str(k): sum(1 for v in views if v["k"] == k) for k in range(6)},
        "views": views,
    }
    with open(os.path.join(HERE, "view_sampling_sec3b.json"), "w") as f:
        f.write(json.dumps(doc, indent=1) + "\n")
