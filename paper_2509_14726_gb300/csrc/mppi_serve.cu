// serving core: filled in with the serving loop
