"""Write the committed benchmark instances (planted, unique solution) as JSON.

    python -m satgen.make_instances [n ...]

Each file satgen/instances/planted_n{n}_s{seed}.json is exactly what
``satgen.planted_instance(n, seed)`` returns; the large sizes are stored because
proving uniqueness at n >= 28 takes minutes of CPU time.
"""

import os
import sys
import time

from satgen import INSTANCE_DIR, planted_instance, save_instance

DEFAULT = [(12, 0), (20, 0), (28, 0), (30, 0), (32, 0)]


def main(argv):
    todo = [(int(a), 0) for a in argv] if argv else DEFAULT
    os.makedirs(INSTANCE_DIR, exist_ok=True)
    for n, seed in todo:
        t0 = time.time()
        inst = planted_instance(n, seed)
        path = os.path.join(INSTANCE_DIR, f"planted_n{n}_s{seed}.json")
        save_instance(inst, path)
        print(f"n={n} seed={seed} m={inst['m']} planted={inst['planted']} "
              f"({time.time() - t0:.1f}s) -> {path}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
