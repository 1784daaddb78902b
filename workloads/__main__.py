"""``python -m workloads`` rewrites the committed 256-run ensemble table."""
from . import write_ensemble_json, ENSEMBLE_JSON

if __name__ == "__main__":
    write_ensemble_json()
    print(ENSEMBLE_JSON)
