"""CPU oracle of the NUMARCK hot path. Test infrastructure only (see numarck_oracle)."""
